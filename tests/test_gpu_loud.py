"""GPU-vs-oracle parity for loud signals.

The subsection "Choices for finite-precision floating point arithmetic and overflow" keeps the
likelihood in log space because loud signals (SNR rho ~ 35 and beyond) overflow raw floating
point.  These tests inject a pulse of <h0|h0> = rho^2 = 1e2, 1e3 and 1e4 (data terms of about
1e2 .. 1e4 near the injection, |lnL_t| up to ~1e5 for prior samples whose template is much louder
than the data) and compare every sample's lnL_t with the FP64 oracle at the path's absolute bar of
1e-3, and ln L_marg at 1e-4, in every precision, through the C ABI.  The fast single-precision
paths alone cannot hold 1e-3 there (their error grows with |D| + A); the FP64 refinement of loud
samples (ile_set_refine) does, and the tests check that it is what runs."""
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


_cache = {}


def _loud_case(orc, rho2, n_near=2048, n_prior=2048):
    if rho2 not in _cache:
        point, theta0 = orc.loud_point(S, S.SEED_BASE + 90, rho2)
        th = orc.loud_samples(S, np.random.default_rng(int(rho2) + 5), theta0, n_near, n_prior)
        _cache[rho2] = (point, th, orc.lnL_t(point, th))
    return _cache[rho2]


@pytest.mark.parametrize("rho2", [1e2, 1e3, 1e4])
@pytest.mark.parametrize("prec", PRECS)
def test_loud_lnL_t_every_sample(ile, orc, prec, rho2):
    point, th, ref = _loud_case(orc, rho2)
    ctx = ile.Context(0, None, prec)
    ctx.set_data(point)
    out = ctx.eval(th)
    err = np.abs(out - ref)
    assert ctx.refine_count() > 0  # the loud samples went through the FP64 path
    assert err.max() < LNL_ATOL, (prec, rho2, err.max(), ref[np.argmax(err)])
    # the magnitudes this covers: data terms near the injection of about rho2
    assert np.abs(ref[:2048]).max() > 0.4 * rho2


@pytest.mark.parametrize("rho2", [1e3, 1e4])
@pytest.mark.parametrize("prec", PRECS)
def test_loud_integral(ile, orc, prec, rho2):
    point, th, ref = _loud_case(orc, rho2)
    rng = np.random.default_rng(3)
    lp = rng.normal(0.0, 0.3, th.shape[1])
    lps = rng.normal(0.0, 0.3, th.shape[1])
    ctx = ile.Context(0, None, prec)
    ctx.set_data(point)
    res, lnl = ctx.integrate(th, ln_prior=lp, ln_ps=lps, want_lnL=True)
    want = orc.mc_stats(ref + lp - lps)
    assert abs(res["ln_L"] - want["ln_I"]) < LNMARG_ATOL, (prec, rho2, res["ln_L"], want["ln_I"])
    assert np.abs(lnl - ref).max() < LNL_ATOL


@pytest.mark.parametrize("prec", PRECS)
def test_fast_path_alone_misses_the_bar_when_loud(ile, orc, prec):
    """Without the refinement the single-precision paths exceed 1e-3 at <h0|h0> = 1e4 -- the reason
    the refinement exists -- and agree with the refined values where the signal is quiet."""
    point, th, ref = _loud_case(orc, 1e4)
    ctx = ile.Context(0, None, prec)
    ctx.set_data(point)
    ctx.set_refine(False)
    fast = ctx.eval(th)
    assert np.abs(fast - ref).max() > LNL_ATOL
    ctx.set_refine(True)
    assert np.abs(ctx.eval(th) - ref).max() < LNL_ATOL


def test_quiet_point_refines_nothing(ile, orc):
    point = S.workload_point(S.FULL)
    th = S.workload_samples(S.FULL, 4096)
    ctx = ile.Context(0, None, "bf16x3")
    ctx.set_data(point)
    out = ctx.eval(th)
    assert ctx.refine_count() == 0
    assert np.abs(out - orc.lnL_t(point, th)).max() < LNL_ATOL


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_loud_adaptive_iteration(ile, orc, prec):
    """The device sampler's samples of a loud point (rho^2 = 1e3), one adaptive iteration: lnL_t of
    every drawn sample against the oracle at 1e-3."""
    point, theta0 = orc.loud_point(S, S.SEED_BASE + 91, 1e3)
    ctx = ile.Context(0, None, prec)
    ctx.set_data(point)
    cfg = ile.make_adapt_cfg(seed=1234, n_per_iter=1 << 14)
    ctx.adapt_run(cfg)
    theta, _, _, lnl = ctx.adapt_last()
    ref = orc.lnL_t(point, theta)
    assert np.abs(lnl - ref).max() < LNL_ATOL
    assert np.abs(ref).max() > 100.0
