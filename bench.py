#!/usr/bin/env python
"""Benchmark of the ILE extrinsic-marginalisation hot path on GB300.

One step = one pass of the hot path over one batch of 2^20 extrinsic samples of the
three-detector (H1, L1, V1), 21-mode, 512-bin, 4096 Hz workload: geometry, mode coefficients,
shifted contraction, quadratic term, time log-sum-exp and the Monte Carlo integral.  Inputs
(seeded, synthetic) are resident in HBM when the timed region starts; the L2 cache is flushed
(a 256 MiB write) between timed steps, outside the per-step CUDA events.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on the host cores
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "extrinsic lnL samples/s on 1 GB300, batched split-prec vs plain, |ΔlnL|≤1e-3"
UNIT = "samples/s"
CONFIG = 1  # 3 detectors, 21 modes, N_t = 512, 2^20 samples


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            ids = [v.strip() for v in vis.split(",") if v.strip()]
            if gpu_index < len(ids):
                gpu_index = ids[gpu_index]
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [r for (t, r) in self.rows if t0 <= t <= t1 + 0.25]
        if not rows:
            rows = [r for (_, r) in self.rows[-3:]]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()) if rows else None}


# ------------------------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    from paper_2210_07912_gb300 import synthetic as S
    oracle.build()
    point = S.config_point(CONFIG)
    cores = os.cpu_count() or 1
    calib = S.config_samples(CONFIG, 256)
    t = time.perf_counter()
    oracle.lnL_t(point, calib, cores)
    per = (time.perf_counter() - t) / 256
    n_step = int(max(256, min(1 << 20, 1.5 / per)))
    all_th = S.config_samples(CONFIG, n_step)
    for _ in range(args.warmup):
        oracle.mc_stats(oracle.lnL_t(point, all_th, cores))
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.mc_stats(oracle.lnL_t(point, all_th, cores))
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = n_step * args.steps / tot
    sample = f"{n_step} of the 2^20 samples per step (FP64 oracle, OpenMP over samples)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(point, 1 << 20, "f64-oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(point, N, prec):
    return {"workload": "ILE extrinsic marginalisation, H1/L1/V1, 21 modes (l<=4), N_t=512 at 4096 Hz, "
                        "2^20 samples per step",
            "n_det": point.n_det, "n_modes": point.n_modes, "n_window": point.n_window, "T_ext": point.T_ext,
            "n_samples": N, "contraction": prec, "l2": "flushed between steps (256 MiB write)"}


def cpu_baseline(point, seconds=12.0):
    import oracle
    from paper_2210_07912_gb300 import synthetic as S
    cores = os.cpu_count() or 1
    calib = S.config_samples(CONFIG, 256)
    t = time.perf_counter()
    oracle.lnL_t(point, calib, cores)
    per = (time.perf_counter() - t) / 256
    n = int(max(256, min(1 << 20, seconds / per)))
    th = S.config_samples(CONFIG, n)
    t = time.perf_counter()
    oracle.mc_stats(oracle.lnL_t(point, th, cores))
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n} of the 2^20 samples of the timed workload, lnL_t + MC integral, FP64"}


# ------------------------------------------------------------------------------------ our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "tf32x3", "bf16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-samples", type=int, default=None,
                    help="samples per step (default 2^20, the benchmarked workload; smaller only for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_2210_07912_gb300 import ile, synthetic as S

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    N = args.n_samples or S.CONFIGS[CONFIG]["n_samples"]
    point = S.make_point(S.SEED_BASE + CONFIG + 1000 * rank, 3, 21, 512, spectrum="decay")
    th_host = S.prior_samples(np.random.default_rng([S.SEED_BASE + CONFIG, rank]), N)
    stream = torch.cuda.Stream()
    ctx = ile.Context(local, stream, args.prec)
    ctx.set_data(point)
    d_th = torch.from_numpy(th_host).cuda()
    d_res = torch.zeros(8, dtype=torch.float64, device="cuda")
    d_lnl = torch.empty(N, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def step():
        ctx.integrate_device(d_th, d_res, lnL_out=d_lnl)

    for _ in range(args.warmup):
        step()
    ctx.sync()

    clocks = ClockSampler(local)
    time.sleep(0.6)
    ctx.profile(True)
    ctx.profile_read()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
        step()
        with torch.cuda.stream(stream):
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    ctx.sync()
    prof = ctx.profile_read()
    ctx.profile(False)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    if dist:
        tt = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
        dist.barrier()
    clk = clocks.summary(t0, t1)
    clocks.stop()
    value = N * args.steps * world / (ms / 1e3)

    # e2e: the public host-pointer API, inputs copied from pinned host memory every step
    pinned = torch.empty((7, N), dtype=torch.float64, pin_memory=True)
    pinned.copy_(torch.from_numpy(th_host))
    th_pinned = pinned.numpy()
    ctx.integrate(th_pinned)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 20))
    t = time.perf_counter()
    for _ in range(e2e_steps):
        res = ctx.integrate(th_pinned)
    e2e_s = time.perf_counter() - t
    if dist:
        tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    e2e_value = N * e2e_steps * world / e2e_s

    if rank == 0:
        pk, pk_kind = peaks()
        K, M, Nt = point.n_det, point.n_modes, point.n_window
        contract_ms, contract_n = prof["contract"]
        per_launch_s = contract_ms / 1e3 / max(1, contract_n)  # one contraction kernel per step
        alg_flops = 4.0 * M * Nt * K * N  # data term of the contraction per launch
        if args.prec == "fp32":
            sm_mhz = pk.get("sm_max_mhz", 2070.0)
            peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x max SM clock
            roof = {"bound": "alu", "achieved": alg_flops / per_launch_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "frac": alg_flops / per_launch_s / 1e12 / peak, "traffic": None,
                    "kernel": "ile_plain_kernel (S3+S5)",
                    "peak_kind": "FP32 CUDA-core FMA rate: 152 SMs x 128 lanes x 2 flop x %.0f MHz" % sm_mhz}
        else:
            peak = pk["bf16_tflops"] * (0.5 if args.prec == "tf32x3" else 1.0)
            roof = {"bound": "tensor", "achieved": alg_flops / per_launch_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "frac": alg_flops / per_launch_s / 1e12 / peak, "traffic": None}
        launches = sum(c for (_, c) in prof.values())
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(point, N, args.prec),
                "roofline": {**roof, "peak_source": pk_kind},
                "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 7 * 8 * N,
                        "d2h_bytes_per_step": 7 * 8},
                "gpu_launches": launches, "clocks": clk,
                "result": {"ln_L_marg": res["ln_L"], "sigma_ln": res["sigma_ln"], "n_eff": res["n_eff"]}}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(point)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
