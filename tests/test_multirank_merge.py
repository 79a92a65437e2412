"""Sharding of the Monte Carlo integral across ranks (CPU, gloo, world size 2).

The path shards over samples (and over intrinsic points) with a single exchange: every rank
reduces its own samples to (max ln w, S1, S2, n, histograms) and the partials are merged.  Each
rank here computes its partial from its half of the samples with the FP64 oracle, the tuples are
all-gathered over gloo, and the library's host merge must reproduce the single-process result
over all samples.  No GPU is used."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

WORLD = 2


def _rank_main(rank, port, out):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2210_07912_gb300 import ile

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    rng = np.random.default_rng(7)
    lnw = rng.normal(0.0, 2.0, 20000) + 50.0  # shared seed: every rank sees the same population
    bins = rng.integers(0, 100, 20000).astype(np.uint8)
    mine = np.arange(20000) % WORLD == rank  # this rank's shard
    st = oracle.mc_stats(lnw[mine])
    h = np.zeros((7, 100))
    h[0] = oracle.hist(lnw[mine], bins[mine]) * st["s1"]  # relative to this shard's max
    part = torch.tensor([st["m"], st["s1"], st["s2"], float(mine.sum())] + list(h.reshape(-1)), dtype=torch.float64)
    gathered = [torch.zeros_like(part) for _ in range(WORLD)]
    dist.all_gather(gathered, part)
    g = torch.stack(gathered).numpy()
    merged = ile.merge_partials(g[:, 0], g[:, 1], g[:, 2], g[:, 3], g[:, 4:].reshape(WORLD, 7, 100))
    full = oracle.mc_stats(lnw)
    ok = (abs(merged["ln_L"] - full["ln_I"]) < 1e-12 and abs(merged["n_eff"] - full["n_eff"]) < 1e-9 * full["n_eff"]
          and abs(merged["sigma_ln"] - full["sigma_ln"]) < 1e-12
          and np.allclose(merged["hist"][0] / merged["hist"][0].sum(), oracle.hist(lnw, bins), rtol=1e-12))
    out[rank] = 1 if ok else 0
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_merge_equals_single_process():
    ctx = mp.get_context("spawn")
    out = ctx.Array("i", [0] * WORLD)
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, port, out)) for r in range(WORLD)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    assert list(out) == [1] * WORLD


def test_merge_ignores_empty_shards_and_rejects_all_empty():
    from paper_2210_07912_gb300 import ile
    d = ile.merge_partials([1.0, -np.inf], [2.0, 0.0], [3.0, 0.0], [5.0, 0.0])
    assert abs(d["ln_L"] - (1.0 + np.log(2.0 / 5.0))) < 1e-15
    with pytest.raises(ile.IleError):
        ile.merge_partials([0.0], [0.0], [0.0], [0.0])
