"""Batched adaptive run (ile_batch_*) through the C ABI (needs a GB300).

Every point of a batch must reproduce, bit for bit, the single-point adaptive run of that point
with the same seed, point id and ranges: the sampler words, the integer tables and the fixed-point
histograms are exact, and a sample's lnL does not depend on which tile or launch evaluates it.
The single-point run is itself checked against the FP64 oracle (test_gpu_adapt); the first
iteration of a batch point is also checked against the oracle directly.
"""
import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

# (K, M, N_t, N): mixed detector sets, mode counts, windows and ragged sample budgets
SHAPES = [(3, 21, 512, 20000), (4, 9, 1024, 5000), (3, 2, 256, 3000), (4, 5, 512, 12000), (3, 9, 256, 700),
          (2, 2, 256, 130)]


@pytest.fixture(scope="module")
def ile():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_07912_gb300 import ile as I
    I.load()
    return I


def _batch_inputs(ile, seed=500):
    points, cfgs = [], []
    for i, (K, M, Nt, N) in enumerate(SHAPES):
        points.append(S.make_point(S.SEED_BASE + seed + i, K, M, Nt, spectrum="decay"))
        mask = [0b11, 0b1011011, 0b11, 0b1000001, 0b11, 0b10][i]
        cfgs.append(ile.make_adapt_cfg(seed=9000 + 17 * i, n_per_iter=N, adapt_mask=mask, point_id=i))
    return points, cfgs


def _single(ile, point, cfg, prec, n_iter):
    ctx = ile.Context(0, None, prec)
    ctx.set_data(point)
    cfg.n_iter = n_iter
    return ctx.adapt_run(cfg)


def _assert_same(a, b, where):
    for key in ("ln_L", "sigma_ln", "n_eff", "ess", "max_lnw", "s1", "s2", "n_total", "n_iter"):
        assert a[key] == b[key], (where, key, a[key], b[key])
    np.testing.assert_array_equal(a["iter_ln_L"], b["iter_ln_L"], err_msg=where)
    np.testing.assert_array_equal(a["cdf"], b["cdf"], err_msg=where)
    np.testing.assert_array_equal(a["hist"], b["hist"], err_msg=where)


def test_batch_equals_single_point_runs(ile):
    points, cfgs = _batch_inputs(ile)
    b = ile.Batch(0, None, "bf16x3")
    res = b.run(points, cfgs, 3)
    for i, (p, c) in enumerate(zip(points, cfgs)):
        _assert_same(res[i], _single(ile, p, c, "bf16x3", 3), f"point {i}")


def test_batch_tf32_equals_single_point_runs(ile):
    """TF32x3 batches run the fused TF32x3 kernel point by point (A operand in TMEM), as a
    single-point run of each point does: the results agree bit for bit."""
    points, cfgs = _batch_inputs(ile, seed=550)
    b = ile.Batch(0, None, "tf32x3")
    res = b.run(points, cfgs, 2)
    for i, (p, c) in enumerate(zip(points, cfgs)):
        _assert_same(res[i], _single(ile, p, c, "tf32x3", 2), f"point {i}")


def test_batch_fp32_path_matches_single_point_runs(ile):
    """The plain FP32 path adds a window bin's two interpolation terms in the order of the
    64-column chunks, whose boundaries follow the tile's first column, i.e. the (atomic) sort
    order within a delay bucket: it agrees with the single-point run to rounding, not bit for bit."""
    points, cfgs = _batch_inputs(ile)
    b = ile.Batch(0, None, "fp32")
    res = b.run(points, cfgs, 1)
    for i, (p, c) in enumerate(zip(points, cfgs)):
        ref = _single(ile, p, c, "fp32", 1)
        assert abs(res[i]["ln_L"] - ref["ln_L"]) < 1e-8, i
        assert abs(res[i]["n_eff"] - ref["n_eff"]) < 1e-8 * ref["n_eff"], i
        assert np.abs(res[i]["cdf"].astype(np.int64) - ref["cdf"].astype(np.int64)).max() <= 16, i


def test_batch_step_get_and_last_samples(ile, orc):
    points, cfgs = _batch_inputs(ile, seed=600)
    b = ile.Batch(0, None, "bf16x3")
    b.set_points(points, cfgs)
    b.step(1)
    res = b.get()
    assert [r["n_iter"] for r in res] == [1] * len(points)
    # the last iteration's samples and likelihoods of one point against the oracle
    theta, lnl = b.last_samples(3)
    ref = orc.lnL_t(points[3], theta[:, :2000])
    assert np.abs(lnl[:2000] - ref).max() < 1e-3
    # first iteration against an independent oracle run (same Philox words)
    lo, hi = ile.default_ranges()
    c = cfgs[0]
    ref = orc.adapt_run(points[0], c.seed, c.n_per_iter, 1, c.adapt_mask, 0.1, lo, hi, point_id=c.point_id)
    assert abs(res[0]["iter_ln_L"][0] - ref["iters"][0]["ln_I"]) < 1e-4
    # more iterations continue the same run; reset restarts it
    b.step(2)
    three = b.get()
    b.reset()
    b.step(3)
    again = b.get()
    for i in range(len(points)):
        _assert_same(three[i], again[i], f"point {i}")


def test_batch_tune_keeps_results(ile):
    points, cfgs = _batch_inputs(ile, seed=700)
    b = ile.Batch(0, None, "bf16x3")
    b.set_points(points, cfgs)
    b.step(2)
    before = b.get()
    t = b.tune(reps=1)
    assert t["a_tmem"] in (0, 1) and t["nb"] in (2, 3, 4) and t["ms"] > 0 and len(t["tried"]) >= 2
    assert 66 <= t["nwcol"] <= (121 if t["a_tmem"] == 0 else 153)
    # per A placement, the widths tried span its admissible range (both ends included), and the
    # choice is the fastest of everything tried
    for a, hi in ((0, 121), (1, 153)):
        widths = sorted({w for aa, _, w, _ in t["tried"] if aa == a})
        assert widths[0] == 66 and widths[-1] == hi and len(widths) >= 8, (a, widths)
    assert min(t["tried"], key=lambda c: c[3])[:3] == (t["a_tmem"], t["nb"], t["nwcol"])
    b.reset()
    b.step(2)
    after = b.get()
    for i in range(len(points)):
        _assert_same(before[i], after[i], f"point {i}")
    # every admissible hand-set configuration gives the same results
    for a_tmem, nb, nwcol, grid in ((0, 2, 72, 40), (1, 4, 153, 152), (1, 2, 80, 37)):
        b.config(nb, nwcol, grid, a_tmem)
        b.reset()
        b.step(2)
        for i, r in enumerate(b.get()):
            _assert_same(before[i], r, f"point {i} (a_tmem {a_tmem}, nb {nb}, nwcol {nwcol}, {grid} CTAs)")


def test_batch_errors(ile):
    points, cfgs = _batch_inputs(ile, seed=800)
    b = ile.Batch(0, None, "bf16x3")
    with pytest.raises(ile.IleError) as e:
        b.step(1)
    assert e.value.status == ile.ILE_E_STATE
    bad = [ile.make_adapt_cfg(seed=1, n_per_iter=0, point_id=0)] + cfgs[1:]
    with pytest.raises(ile.IleError) as e:
        b.set_points(points, bad)
    assert e.value.status == ile.ILE_E_ARG
    b.set_points(points, cfgs)
    with pytest.raises(ile.IleError) as e:
        b.get(len(points) - 1, 2)
    assert e.value.status == ile.ILE_E_ARG
    with pytest.raises(ile.IleError) as e:
        b.config(2, 10, 152)  # window narrower than one chunk
    assert e.value.status == ile.ILE_E_ARG
    with pytest.raises(ile.IleError) as e:
        b.config(2, 129, 152, 0)  # wider than the shared-memory placement's 128-column buffers allow
    assert e.value.status == ile.ILE_E_ARG
    with pytest.raises(ile.IleError) as e:
        b.config(2, 100, 152, 2)  # no such placement
    assert e.value.status == ile.ILE_E_ARG
    f = ile.Batch(0, None, "fp32")
    f.set_points(points[:2], cfgs[:2])
    with pytest.raises(ile.IleError) as e:
        f.tune()
    assert e.value.status == ile.ILE_E_STATE
