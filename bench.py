#!/usr/bin/env python
"""Benchmark of the ILE extrinsic-marginalisation hot path on GB300.

One step = one iteration of the adaptive Monte Carlo integrator over 2^20 extrinsic samples of
the three-detector (H1, L1, V1), 21-mode, 512-bin, 4096 Hz workload, every stage on the device:
Philox sampling from the adaptive histograms (S0), geometry and mode coefficients (S1, S2), the
shifted contraction (S3, split-precision BF16x3 tensor cores by default), the quadratic term
(S4), the time log-sum-exp (S5), the Monte Carlo integral and the histogram refit (S6).  The
intrinsic point's Q/U/V are resident in HBM when the timed region starts; the L2 cache is flushed
(a 256 MiB write) between timed steps, outside the per-step CUDA events.  The plain FP32
CUDA-core path is timed on the same workload for comparison.

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
WORKLOAD = "hlv_m21_nt512"  # 3 detectors, 21 modes, N_t = 512, 2^20 samples (synthetic.FULL)
SEED_ADAPT = 2210079121  # Philox key of the benchmarked sampler


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


# ------------------------------------------------------------------------------------ workload
def workload_config(point, N, prec):
    return {"workload": "ILE extrinsic marginalisation, one adaptive MC iteration: H1/L1/V1, 21 modes "
                        "(l<=4), N_t=512 at 4096 Hz, 2^20 samples per step",
            "n_det": point.n_det, "n_modes": point.n_modes, "n_window": point.n_window, "T_ext": point.T_ext,
            "n_samples": N, "contraction": prec, "adaptive_dims": "ra, sin dec (100-bin histograms)",
            "l2": "flushed between steps (256 MiB write)"}


def oracle_step(point, N, it, seed=SEED_ADAPT, nthreads=0):
    """One adaptive iteration in the FP64 oracle (sampling, lnL_t, MC sums, histogram refit) on N
    samples; returns the elapsed wall time."""
    import oracle
    from paper_2210_07912_gb300 import ile
    lo, hi = ile.default_ranges()
    t = time.perf_counter()
    oracle.adapt_run(point, seed, N, 1, 0b11, 0.1, lo, hi, point_id=0, nthreads=nthreads, iter0=it)
    return time.perf_counter() - t



def cpu_sample_size(point, seconds, cores):
    from paper_2210_07912_gb300 import synthetic as S
    import oracle
    calib = S.workload_samples(WORKLOAD, 512)
    t = time.perf_counter()
    oracle.lnL_t(point, calib, cores)
    per = (time.perf_counter() - t) / 512
    return int(max(512, min(1 << 20, seconds / per)))


def oracle_error(ctx, point, n=2048):
    """lnL_t of a random subset of the context's last iteration (device samples, device values)
    against the FP64 oracle evaluated on the same samples."""
    import numpy as np
    import oracle
    theta, _, _, lnl = ctx.adapt_last()
    idx = np.random.default_rng(11).choice(theta.shape[1], min(n, theta.shape[1]), replace=False)
    ref = oracle.lnL_t(point, np.ascontiguousarray(theta[:, idx]))
    d = np.abs(lnl[idx] - ref)
    return {"max_abs_dlnL_t": float(d.max()), "rms_dlnL_t": float(np.sqrt(np.mean(d * d))),
            "samples_checked": int(idx.size), "bar": 1e-3,
            "what": "lnL_t of random samples of the last device iteration vs the FP64 oracle on the same samples"}


def loud_error(ile, S, local, prec, rho2s=(1e3, 1e4)):
    """lnL_t of injections of <h0|h0> = rho2 (2048 samples near the injection, 2048 from the prior)
    against the FP64 oracle: the loud regime of App. "Choices for finite-precision floating point
    arithmetic and overflow", through the default path (loud samples refined in FP64)."""
    import oracle
    out = []
    for rho2 in rho2s:
        point, theta0 = oracle.loud_point(S, S.SEED_BASE + 90, rho2)
        th = oracle.loud_samples(S, np.random.default_rng(int(rho2) + 5), theta0, 2048, 2048)
        ref = oracle.lnL_t(point, th)
        ctx = ile.Context(local, None, prec)
        ctx.set_data(point)
        d = np.abs(ctx.eval(th) - ref)
        out.append({"rho2": rho2, "max_abs_dlnL_t": float(d.max()), "rms_dlnL_t": float(np.sqrt(np.mean(d * d))),
                    "max_abs_lnL_t": float(np.abs(ref).max()), "samples_checked": int(d.size),
                    "samples_refined": ctx.refine_count(), "bar": 1e-3})
        ctx.close()
    return out


def error_vs_data_term(ile, S, local, precs=("bf16x3", "tf32x3", "fp32"), n=1024):
    """|lnL_t - oracle| of each precision binned by the sample's largest |data term|
    max_j |Re sum_k (D_ref/D) conj(F_k Y) Q_k(j)|: the benchmarked point's prior samples plus
    injections of <h0|h0> = 1e2, 1e3, 1e4 (n samples near each injection, n from the prior).  For
    every bin: the raw single-precision path (FP64 refinement of loud samples off) and the shipped
    path (refinement on)."""
    import oracle
    cases = [(S.workload_point(WORKLOAD), S.workload_samples(WORKLOAD, 2 * n))]
    for rho2 in (1e2, 1e3, 1e4):
        point, theta0 = oracle.loud_point(S, S.SEED_BASE + 90, rho2)
        cases.append((point, oracle.loud_samples(S, np.random.default_rng(int(rho2) + 5), theta0, n, n)))
    edges = [0.0, 1.0, 10.0, 100.0, 1e3, 1e4, 1e5]
    mags, refs = [], []
    for point, th in cases:
        mag = np.empty(th.shape[1])
        for i in range(th.shape[1]):
            _, data, _ = oracle.lnL_grid(point, th[:, i])
            mag[i] = np.abs(data).max()
        mags.append(mag)
        refs.append(oracle.lnL_t(point, th))
    mag = np.concatenate(mags)
    bins = np.digitize(mag, edges[1:-1])
    out = {"bin_edges_abs_data_term": edges, "samples_per_bin": np.bincount(bins, minlength=len(edges) - 1).tolist()}
    for prec in precs:
        res = {}
        for refine in (False, True):
            errs = []
            for (point, th), ref in zip(cases, refs):
                ctx = ile.Context(local, None, prec)
                ctx.set_data(point)
                ctx.set_refine(refine)
                errs.append(np.abs(ctx.eval(th) - ref))
                ctx.close()
            err = np.concatenate(errs)
            res["refined" if refine else "raw"] = {
                "max_abs_dlnL_t": [float(err[bins == b].max()) if np.any(bins == b) else None
                                   for b in range(len(edges) - 1)],
                "rms_dlnL_t": [float(np.sqrt(np.mean(err[bins == b] ** 2))) if np.any(bins == b) else None
                               for b in range(len(edges) - 1)]}
        out[prec] = res
    return out


def cpu_baseline(point, seconds=12.0):
    cores = os.cpu_count() or 1
    n = cpu_sample_size(point, seconds, cores)
    dt = oracle_step(point, n, 0, nthreads=cores)
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one adaptive iteration on {n} of the 2^20 samples (same seed and tables), FP64, "
                      f"OpenMP over samples"}


# ------------------------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    from paper_2210_07912_gb300 import synthetic as S
    oracle.build()
    point = S.workload_point(WORKLOAD)
    cores = os.cpu_count() or 1
    n_step = cpu_sample_size(point, 1.5, cores)
    for w in range(args.warmup):
        oracle_step(point, n_step, w, nthreads=cores)
    tot = sum(oracle_step(point, n_step, args.warmup + i, nthreads=cores) for i in range(args.steps))
    value = n_step * args.steps / tot
    sample = f"{n_step} of the 2^20 samples per step (one adaptive iteration, FP64 oracle, OpenMP over samples)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(point, 1 << 20, "f64-oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------ our arm
def profile_traffic(kernel_files, prec):
    """DRAM bytes per launch of the contraction kernel from the committed ncu summary, if it was
    taken on the current source of that kernel (else None).  kernel_files: the kernel's source
    files; the two headers every kernel is compiled with are added."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2210_07912_gb300", "csrc")
    srcs = [os.path.join(csrc, f) for f in (*kernel_files, "ile_tcgen05.cuh", "ile_internal.cuh")]
    summ = os.path.join(ROOT, "profiles", f"contract_{prec}_c1.md")
    if not (all(os.path.exists(f) for f in srcs) and os.path.exists(summ)):
        return None, None
    h = hashlib.sha256()
    for f in srcs:
        h.update(open(f, "rb").read())
    digest = h.hexdigest()[:16]
    vals = {}
    for line in open(summ):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256_16") != digest:
        return None, digest
    try:
        return float(vals["dram_bytes_per_launch_full"]), digest
    except (KeyError, ValueError):
        return None, digest


def profile_fraction(kernel_file, prec, metric):
    """A percentage metric (as a fraction) of the committed ncu capture of the contraction kernel,
    if it was taken on the current source (else None)."""
    traffic, digest = profile_traffic(kernel_file, prec)
    if traffic is None:
        return None
    summ = os.path.join(ROOT, "profiles", f"contract_{prec}_c1.md")
    for line in open(summ):
        if line.strip().startswith(f"- {metric}:"):
            try:
                return float(line.split(":", 1)[1].split()[0]) / 100.0
            except (IndexError, ValueError):
                return None
    return None


def profile_tensor_active(kernel_file, prec):
    """Tensor-pipe activity (fraction) of the committed capture of the contraction kernel."""
    return profile_fraction(kernel_file, prec, "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active")


def batch_bench(ile, S, local, flush, iters=5, n_points=512, plain_iters=5):
    """The mixed batch: n_points intrinsic points (M in {2,5,9,21}, K in {3,4}, N_t in
    {256,512,1024}, 2^U(14,20) samples each), `iters` adaptive iterations, tiles chosen by the
    autotuner, every iteration one CUDA-graph launch; the same batch with the plain FP32
    contraction for comparison (`plain_iters` iterations)."""
    import torch
    descs = S.batch_descs(n_points=n_points)
    points = [S.make_point(d["seed"], d["n_det"], d["n_modes"], d["n_window"], spectrum="decay") for d in descs]
    cfgs = [ile.make_adapt_cfg(seed=SEED_ADAPT + 7 * i, n_per_iter=d["n_samples"], adapt_mask=0b11, point_id=i)
            for i, d in enumerate(descs)]
    n_iter_samples = sum(d["n_samples"] for d in descs)

    # algorithmic data-term flops of one iteration (4 M N_t K per sample, every point)
    alg_flops = sum(4.0 * d["n_modes"] * d["n_window"] * d["n_det"] * d["n_samples"] for d in descs)

    def timed(prec, n_it, tune):
        st = torch.cuda.Stream()
        b = ile.Batch(local, st, prec)
        b.set_points(points, cfgs)
        t = b.tune(reps=3) if tune else None
        b.reset()
        b.step(1)  # warm-up iteration (graph instantiation), then restart the run
        b.get()
        b.reset()
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        b.step(n_it)
        e1.record(st)
        res = b.get()
        e1.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        b.close()
        return dt, res, t

    dt, res, tuning = timed("bf16x3", iters, True)
    peak = peaks()[0]["bf16_tflops"]
    achieved = alg_flops * iters / dt / 1e12
    line = {"workload": f"{n_points} intrinsic points (M in {{2,5,9,21}}, K in {{3,4}}, N_t in {{256,512,1024}}, "
                        f"2^U(14,20) samples per point per iteration), {iters} adaptive iterations",
            "n_points": n_points, "samples_per_iteration": n_iter_samples, "iterations": iters,
            "value": n_iter_samples * iters / dt, "unit": UNIT, "s_per_iteration": dt / iters,
            "contraction": "bf16x3, one persistent launch per iteration", "tuning": tuning,
            "ln_L_marg_first_points": [r["ln_L"] for r in res[:4]],
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "what": "algorithmic data-term flops of every point / whole iteration time (sampling, "
                                 "sort, MC sums and histograms included), against the measured dense bf16 peak"},
            "timing": "CUDA events on the batch's stream around step(iterations) (graph launches)"}
    if plain_iters:
        pdt, _, _ = timed("fp32", plain_iters, False)
        line["plain_fp32"] = {"value": n_iter_samples * plain_iters / pdt, "s_per_iteration": pdt / plain_iters,
                              "iterations": plain_iters}
        line["speedup_vs_plain"] = line["value"] / line["plain_fp32"]["value"]
    return line


def dmarg_bench(ile, point, cfg, N, local, stream, flush, prec, steps=20):
    """The benchmarked adaptive iteration with the likelihood marginalised over distance (the
    D^2 prior on [100, 1000] Mpc through the device lookup tables; D not sampled adaptively)."""
    import torch
    ctx = ile.Context(local, stream, prec)
    ctx.set_data(point)
    t = time.perf_counter()
    ctx.set_distance_marginalization(True, 100.0, 1000.0)
    t_tables = time.perf_counter() - t
    ctx.adapt_init(cfg)
    ctx.adapt_step(3)
    ctx.sync()
    ctx.profile(True)
    ctx.profile_read()
    ms = 0.0
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        ctx.adapt_step(1)
        with torch.cuda.stream(stream):
            b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    prof = ctx.profile_read()
    res = ctx.adapt_get()
    ctx.close()
    return {"workload": "the benchmarked adaptive iteration (H1/L1/V1, 21 modes, N_t=512, 2^20 samples) with the "
                        "likelihood marginalised over D (D^2 prior on [100, 1000] Mpc)",
            "value": N * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "contraction": prec,
            "stage_ms_per_step": {k: v[0] / steps for k, v in prof.items() if v[1]},
            "table_build_s": t_tables, "ln_L_marg": res["ln_L"], "sigma_ln": res["sigma_ln"]}


def adjoint_bench(ile, S, local, stream, flush, steps=10, prec="bf16x3"):
    """Gradient of ln L_marg-style weighted sums: ile_eval_grad over 2^18 samples of the
    3-detector, 21-mode, 512-bin point, all outputs (theta, Q, U, V), FP64 sums.  prec bf16x3: the
    data term comes from the fused tensor-core forward kernel; fp32: recomputed on CUDA cores."""
    import torch
    point = S.workload_point(S.GRAD)
    N = S.WORKLOADS[S.GRAD]["n_samples"]
    th = torch.tensor(S.workload_samples(S.GRAD), device="cuda")
    g = torch.tensor(np.random.default_rng(4).normal(size=N), device="cuda")
    K, M, T = point.Q.shape
    gs = torch.empty_like(th)
    gQ = torch.empty((K, M, T, 2), dtype=torch.float64, device="cuda")
    gU = torch.empty((K, M, M, 2), dtype=torch.float64, device="cuda")
    gV = torch.empty_like(gU)
    ctx = ile.Context(local, stream, prec)
    ctx.set_data(point)
    for _ in range(3):
        ctx.eval_grad_device(th, g, gs, gQ, gU, gV)
    ctx.sync()
    ctx.profile(True)
    ctx.profile_read()
    ms = 0.0
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        ctx.eval_grad_device(th, g, gs, gQ, gU, gV)
        with torch.cuda.stream(stream):
            b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    prof = ctx.profile_read()
    ctx.sync()
    ctx.close()
    flops = 16.0 * M * point.n_window * K * N  # forward recompute + E + slope + dQ contractions
    return {"workload": "gradient of sum_n g_n lnL_t(n) w.r.t. theta (7 x 2^18), Q, U, V: H1/L1/V1, 21 modes, "
                        "N_t=512, 2^18 samples", "value": N * steps / (ms / 1e3), "unit": UNIT,
            "ms_per_call": ms / steps, "stage_ms_per_call": {k: v[0] / steps for k, v in prof.items() if v[1]},
            "algorithmic_tflops": flops / (ms / steps / 1e3) / 1e12,
            "arithmetic": ("data term from the fused BF16x3 tensor-core kernel, E / slope and dQ contractions as "
                           "BF16x3 tcgen05 GEMMs, chain rule on fp32 CUDA cores, fp64 sums"
                           if prec == "bf16x3" else "fp32 CUDA cores, fp64 sums"), "precision": prec}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["fp32", "tf32x3", "bf16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-point batched run")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (gradient) measurement")
    ap.add_argument("--no-dmarg", action="store_true", help="skip the distance-marginalised measurement")
    ap.add_argument("--batch-points", type=int, default=512)
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

    N = args.n_samples or S.WORKLOADS[WORKLOAD]["n_samples"]
    # replicas: every rank integrates its own intrinsic point
    c = S.WORKLOADS[WORKLOAD]
    point = S.make_point(S.SEED_BASE + c["seed"] + 1000 * rank, c["n_det"], c["n_modes"], c["n_window"],
                         spectrum=c["spectrum"])
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    cfg = ile.make_adapt_cfg(seed=SEED_ADAPT + rank, n_per_iter=N, adapt_mask=0b11, point_id=rank)

    def timed(prec, steps, profile):
        ctx = ile.Context(local, stream, prec)
        ctx.set_data(point)
        ctx.adapt_init(cfg)
        ctx.adapt_step(args.warmup)
        ctx.sync()
        ctx.profile(profile)
        if profile:
            ctx.profile_read()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.time()
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
                evs[i][0].record(stream)
            ctx.adapt_step(1)
            with torch.cuda.stream(stream):
                evs[i][1].record(stream)
        torch.cuda.synchronize()
        t1 = time.time()
        res = ctx.adapt_get()
        prof = ctx.profile_read() if profile else None
        ctx.profile(False)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        if dist:
            tt = torch.tensor([ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms = float(tt.item())
        return ms, prof, res, (t0, t1), ctx

    clocks = ClockSampler(local)
    time.sleep(0.6)
    ms, prof, res, (t0, t1), ctx = timed(args.prec, args.steps, True)
    clk = clocks.summary(t0, t1)
    clocks.stop()
    value = N * args.steps * world / (ms / 1e3)

    plain = None
    if not args.no_plain and args.prec != "fp32":
        pms, _, _, _, pctx = timed("fp32", max(3, min(args.steps, 10)), False)
        psteps = max(3, min(args.steps, 10))
        plain = {"value": N * psteps * world / (pms / 1e3), "ms_per_step": pms / psteps, "contraction": "fp32"}
        pctx.close()
    # the other split-precision variant of the same workload (config c2 asks for both)
    variants = {}
    if not args.no_plain:  # every rank times it (the timing takes a barrier); rank 0 reports
        for vp in ("bf16x3", "tf32x3"):
            if vp == args.prec:
                vctx, vms, vprof, vsteps = ctx, ms, prof, args.steps
            else:
                vsteps = max(3, min(args.steps, 10))
                vms, vprof, _, _, vctx = timed(vp, vsteps, True)
            cm, cn = vprof["contract"]
            variants[vp] = {"value": N * vsteps / (vms / 1e3), "ms_per_step": vms / vsteps,
                            "contract_ms_per_step": cm / vsteps,
                            "error_vs_oracle": None if (args.no_cpu_baseline or rank != 0)
                            else oracle_error(vctx, point)}
            if vctx is not ctx:
                vctx.close()

    # e2e: a user's full evaluation of one intrinsic point through the public API every step --
    # upload the point (host arrays), set up the sampler, one iteration, read the result back
    e2e_steps = max(3, min(args.steps, 20))
    ctx.set_data(point)
    ctx.adapt_init(cfg)
    ctx.adapt_step(1)
    ctx.adapt_get(raw=True)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.set_data(point)
        ctx.adapt_init(cfg)
        ctx.adapt_step(1)
        r = ctx.adapt_get(raw=True)
    e2e_s = time.perf_counter() - t
    if dist:
        tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    e2e_value = N * e2e_steps * world / e2e_s
    K, M, Nt, T = point.n_det, point.n_modes, point.n_window, point.T_ext
    h2d = 8 * 2 * K * M * T + 8 * 2 * 2 * K * M * M + 8 * (12 * K) + 4 * 2 * M + 8 * 2 * 7 + 64

    if rank == 0:
        pk, pk_kind = peaks()
        contract_ms, contract_n = prof["contract"]
        per_launch_s = contract_ms / 1e3 / max(1, contract_n)
        alg_flops = 4.0 * M * Nt * K * N  # data term of the contraction, per launch
        if args.prec == "fp32":
            sm_mhz = pk.get("sm_max_mhz", 2070.0)
            peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
            roof = {"bound": "alu", "kernel": "ile_plain_kernel (S3+S5)",
                    "peak_kind": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x %.0f MHz" % sm_mhz}
            kfile = ("ile_plain.cu",)
        else:
            peak = pk["bf16_tflops"] * (0.5 if args.prec == "tf32x3" else 1.0)
            roof = {"bound": "tensor",
                    "kernel": "ile_tc2_kernel (S1-S5 fused, BF16x3, A operand in shared memory)"
                    if args.prec == "bf16x3" else "ile_tc2_kernel (S1-S5 fused, TF32x3, A operand in TMEM)",
                    "peak_kind": "measured dense bf16 (burst)" + (" x 1/2 for tf32" if args.prec == "tf32x3" else "")}
            kfile = ("ile_tc2_kernel.cuh", "ile_tc2.cu" if args.prec == "bf16x3" else "ile_tc3.cu")
        traffic, _ = profile_traffic(kfile, args.prec)
        achieved = alg_flops / per_launch_s / 1e12
        roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic, "tensor_pipe_active_ncu": profile_tensor_active(kfile, args.prec),
                     # the kernel's actual limiter: instruction issue of its math warps
                     "issue_active_ncu": profile_fraction(
                         kfile, args.prec, "smsp__issue_active.avg.pct_of_peak_sustained_active"),
                     "algorithmic_flops_per_launch": alg_flops,
                     "launch_ms": per_launch_s * 1e3, "peak_source": pk_kind})
        launches = sum(c for (_, c) in prof.values())  # kernels launched by the library in the timed steps
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3" if args.prec == "bf16x3" else "f32",
                "data": "synthetic", "config": workload_config(point, N, args.prec),
                "roofline": roof,
                "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
                "plain_fp32": plain,
                "speedup_vs_plain": (value / plain["value"]) if plain else None,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": 8 * 20 + 8 * 2 * 64 + 8 * 7 * 101 + 8 * 7 * 100,
                        "what": "set_data (host arrays) + adapt_init + one iteration + result read-back"},
                "gpu_launches": launches, "clocks": clk,
                "result": {"ln_L_marg": res["ln_L"], "sigma_ln": res["sigma_ln"], "n_eff": res["n_eff"],
                           "iterations": res["n_iter"]}}
        if variants:
            line["split_variants"] = variants
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(point)
            line["error_vs_oracle"] = oracle_error(ctx, point)
            line["error_vs_oracle_loud"] = loud_error(ile, S, local, args.prec)
            line["split_error_vs_data_term"] = error_vs_data_term(ile, S, local)
        if not args.no_adjoint:
            line["adjoint"] = adjoint_bench(ile, S, local, stream, flush, prec=args.prec)
        if not args.no_dmarg:
            line["distance_marginalised"] = dmarg_bench(ile, point, cfg, N, local, stream, flush, args.prec)
        if not args.no_batch:
            line["batch"] = batch_bench(ile, S, local, flush, n_points=args.batch_points)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
