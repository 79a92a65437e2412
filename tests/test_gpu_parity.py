"""GPU-vs-oracle parity of the ILE hot path through the C ABI (needs a GB300).

Bar: per-sample lnL and lnL_t within 1e-3 absolute of the FP64 oracle, ln L_marg within 1e-4
(the tolerances the path is specified to), on the same seeded inputs.  Small cases compare every
element and span several sample tiles plus a ragged tail; the full 2^20-sample workload is
compared on a random subset the oracle computes one by one.
"""
import math

import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

LNL_ATOL = 1e-3
LNMARG_ATOL = 1e-4
PRECS = ["fp32", "tf32x3", "bf16x3"]


@pytest.fixture(scope="module")
def ile():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_07912_gb300 import ile as I
    I.load()
    return I


def _ctx(ile, point, prec="fp32"):
    c = ile.Context(0, None, prec)
    c.set_data(point)
    return c


@pytest.mark.parametrize("prec", PRECS)
def test_grid_matches_oracle_small_point(ile, orc, prec):
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 300)  # 4 full tiles of 64 + a ragged tail
    ctx = _ctx(ile, point, prec)
    grid = ctx.eval(th, grid=True)
    for n in range(th.shape[1]):
        ref, _, _ = orc.lnL_grid(point, th[:, n])
        err = np.abs(grid[n] - ref).max()
        assert err < LNL_ATOL, (n, err)


@pytest.mark.parametrize("prec", PRECS)
def test_lnL_t_matches_oracle_small_point_all_samples(ile, orc, prec):
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL)
    ctx = _ctx(ile, point, prec)
    got = ctx.eval(th)
    ref = orc.lnL_t(point, th)
    err = np.abs(got - ref)
    assert err.max() < LNL_ATOL, err.max()


@pytest.mark.parametrize("prec", PRECS)
def test_lnL_t_matches_oracle_full_shape_1000_samples(ile, orc, prec):
    point = S.workload_point(S.FULL)
    th = S.workload_samples(S.FULL, 1000)
    ctx = _ctx(ile, point, prec)
    got = ctx.eval(th)
    ref = orc.lnL_t(point, th)
    assert np.abs(got - ref).max() < LNL_ATOL


@pytest.mark.parametrize("prec", PRECS)
def test_lnL_t_full_size_sampled(ile, orc, prec):
    """2^20 samples on the device (the benchmarked launch); 2048 random ones checked by the oracle."""
    point = S.workload_point(S.FULL)
    th = S.workload_samples(S.FULL)
    ctx = _ctx(ile, point, prec)
    got = ctx.eval(th)
    idx = np.random.default_rng(3).choice(th.shape[1], 2048, replace=False)
    ref = orc.lnL_t(point, th[:, idx])
    assert np.abs(got[idx] - ref).max() < LNL_ATOL
    assert np.all(np.isfinite(got))


@pytest.mark.parametrize("prec", PRECS)
# (4, 20, 130): the TF32x3 A operand of the fused kernel at its 320-column limit; (4, 21, 256): beyond it
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 3, 7), (4, 9, 33), (3, 21, 1024), (2, 5, 300), (4, 20, 130),
                                   (4, 21, 256)])
def test_odd_shapes(ile, orc, shape, prec):
    K, M, Nt = shape
    point = S.make_point(77 + K * M + Nt, K, M, Nt, spectrum="random")
    th = S.prior_samples(np.random.default_rng(K * 100 + M), 130)
    ctx = _ctx(ile, point, prec)
    got = ctx.eval(th)
    ref = orc.lnL_t(point, th)
    assert np.abs(got - ref).max() < LNL_ATOL


@pytest.mark.parametrize("prec", PRECS)
def test_integrate_matches_oracle(ile, orc, prec):
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL)
    rng = np.random.default_rng(4)
    lnp = rng.normal(0, 0.3, th.shape[1])
    lnps = rng.normal(0, 0.3, th.shape[1])
    ctx = _ctx(ile, point, prec)
    res, lnl = ctx.integrate(th, lnp, lnps, want_lnL=True)
    ref_lnl = orc.lnL_t(point, th)
    st = orc.mc_stats(ref_lnl + lnp - lnps)
    assert abs(res["ln_L"] - st["ln_I"]) < LNMARG_ATOL
    assert abs(res["n_eff"] - st["n_eff"]) < 1e-3 * st["n_eff"]
    assert abs(res["ess"] - st["ess"]) < 1e-3 * st["ess"]
    assert abs(res["sigma_ln"] - st["sigma_ln"]) < 1e-3 * st["sigma_ln"] + 1e-9
    assert np.abs(lnl - ref_lnl).max() < LNL_ATOL


@pytest.mark.parametrize("prec", PRECS)
def test_integrate_full_size(ile, orc, prec):
    """ln L_marg over 2^20 samples: the device reduction equals the oracle reduction of the device
    lnL_t, and the device lnL_t is within tolerance of the oracle on a random subset."""
    point = S.workload_point(S.FULL)
    th = S.workload_samples(S.FULL)
    ctx = _ctx(ile, point, prec)
    res, lnl = ctx.integrate(th, want_lnL=True)
    st = orc.mc_stats(lnl)
    assert abs(res["ln_L"] - st["ln_I"]) < 1e-6
    idx = np.random.default_rng(5).choice(th.shape[1], 1024, replace=False)
    assert np.abs(lnl[idx] - orc.lnL_t(point, th[:, idx])).max() < LNL_ATOL
    # a per-sample error bounded by e shifts ln L_marg by at most e
    assert abs(res["ln_L"] - st["ln_I"]) < LNMARG_ATOL


def test_device_pointer_path(ile, orc):
    import torch
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 5000)
    ctx = _ctx(ile, point)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    d_th = torch.from_numpy(th).cuda()
    d_out = torch.empty(th.shape[1], dtype=torch.float64, device="cuda")
    d_res = torch.empty(8, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ctx.eval_device(d_th, d_out)
    ctx.integrate_device(d_th, d_res)
    ctx.sync()
    ref = orc.lnL_t(point, th)
    assert np.abs(d_out.cpu().numpy() - ref).max() < LNL_ATOL
    assert abs(d_res[0].item() - orc.mc_stats(ref)["ln_I"]) < LNMARG_ATOL


def test_error_paths(ile):
    point = S.workload_point(S.SMALL)
    c = ile.Context(0)
    with pytest.raises(ile.IleError) as e:
        c.eval(S.workload_samples(S.SMALL, 4))
    assert e.value.status == ile.ILE_E_STATE
    c.set_data(point)
    assert c.eval(np.zeros((7, 0))).shape == (0,)
    th = S.workload_samples(S.SMALL, 100)
    th[6, 17] = 0.05  # coalescence time far outside the window
    with pytest.raises(ile.IleError) as e:
        c.eval(th)
    assert e.value.status == ile.ILE_E_RANGE
    th = S.workload_samples(S.SMALL, 100)
    th[0, 3] = np.nan
    with pytest.raises(ile.IleError) as e:
        c.eval(th)
    assert e.value.status == ile.ILE_E_NONFINITE
    # the context is still usable afterwards
    good = S.workload_samples(S.SMALL, 10)
    assert np.all(np.isfinite(c.eval(good)))
    bad = S.Point(**{**point.__dict__, "lm": np.array([[2, 2], [2, 2]], np.int32)})
    with pytest.raises(ile.IleError) as e:
        c.set_data(bad)
    assert e.value.status == ile.ILE_E_ARG


def _half_integer_clear(orc, point, th, margin=1e-3):
    """Samples whose window starts are at least `margin` samples away from a half-integer in
    every detector: there the nearest-sample choice does not depend on FP32 vs FP64 rounding."""
    keep = np.ones(th.shape[1], bool)
    for n in range(th.shape[1]):
        for k in range(point.n_det):
            dt = orc.delay(point.det_pos[k], th[0, n], th[1, n], point.gmst)
            x = (th[6, n] - point.n_window / 2 / point.fs + dt - point.t_start) * point.fs
            if abs((x - np.floor(x)) - 0.5) < margin:
                keep[n] = False
    return th[:, keep]


@pytest.mark.parametrize("prec", PRECS)
def test_nearest_sample_mode_matches_oracle(ile, orc, prec):
    """ILE_NEAREST (Q at the nearest sample) against the oracle's brute-force-pinned nearest mode,
    every sample of the small point and 2000 of the full-shape point."""
    for name, N in ((S.SMALL, 2000), (S.FULL, 2000)):
        point = S.workload_point(name)
        th = _half_integer_clear(orc, point, S.workload_samples(name, N))
        ctx = ile.Context(0, None, prec)
        ctx.set_data(point)
        got = ctx.eval(th, nearest=True)
        ref = orc.lnL_t(point, th, nearest=True)
        assert np.abs(got - ref).max() < 1e-3, (name, prec)
        # and the nearest mode is a different function from the interpolated one
        assert np.abs(ctx.eval(th) - ref).max() > 1e-6


def test_set_data_nonfinite_q(ile, orc):
    """A non-finite Q is found on the device while Q is converted: ILE_E_NONFINITE, and the
    context then has no point until the next successful ile_set_data (which evaluates as usual)."""
    point = S.workload_point(S.SMALL)
    c = ile.Context(0)
    q = point.Q.copy()
    q[1, 0, 7] = complex(np.inf, 0.0)
    with pytest.raises(ile.IleError) as e:
        c.set_data(S.Point(**{**point.__dict__, "Q": q}))
    assert e.value.status == ile.ILE_E_NONFINITE
    th = S.workload_samples(S.SMALL, 64)
    with pytest.raises(ile.IleError) as e:
        c.eval(th)
    assert e.value.status == ile.ILE_E_STATE
    c.set_data(point)
    assert np.abs(c.eval(th) - orc.lnL_t(point, th)).max() < 1e-3
