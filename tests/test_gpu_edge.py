"""Edge cases of the hot path against the oracle, through the C ABI (needs a GB300): a single
sample, the largest launch the adaptive API accepts (2^23 samples per iteration), samples whose
time windows touch both ends of the extended Q series, and the degenerate inputs of the method
(no data, Q = 0: the likelihood is the quadratic term alone; no signal model power, U = V = 0:
the data term alone)."""
import math

import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

LNL_ATOL = 1e-3
PRECS = ["fp32", "tf32x3", "bf16x3"]
C_SI = 299792458.0


@pytest.fixture(scope="module")
def ile():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_07912_gb300 import ile as I
    I.load()
    return I


def _ctx(ile, point, prec):
    c = ile.Context(0, None, prec)
    c.set_data(point)
    return c


@pytest.mark.parametrize("prec", PRECS)
def test_single_sample(ile, orc, prec):
    point = S.workload_point(S.FULL)
    th = S.workload_samples(S.FULL, 1)
    got = _ctx(ile, point, prec).eval(th)
    assert got.shape == (1,)
    assert abs(got[0] - orc.lnL_t(point, th)[0]) < LNL_ATOL


def _toward(v, gmst):
    """(ra, dec) of the unit vector v (Earth-fixed) at the given GMST."""
    v = np.asarray(v, float) / np.linalg.norm(v)
    return (gmst - math.atan2(-v[1], v[0])) % (2 * math.pi), math.asin(v[2])


@pytest.mark.parametrize("prec", PRECS)
def test_windows_at_both_ends_of_the_series(ile, orc, prec):
    """Sky directions along and against each detector's position (largest delays) with t_c at both
    ends of its range: the windows reach the first and last columns of Q, no range error."""
    point = S.workload_point(S.FULL)
    rng = np.random.default_rng(11)
    cols = []
    for r in point.det_pos:
        for sgn in (1.0, -1.0):
            ra, dec = _toward(sgn * r, point.gmst)
            for tc in (-point.tc_max, point.tc_max):
                cols.append([ra, dec, rng.uniform(0, math.pi), rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi),
                             rng.uniform(100, 1000), tc])
    th = np.array(cols).T.copy()
    got = _ctx(ile, point, prec).eval(th)
    ref = orc.lnL_t(point, th)
    assert np.abs(got - ref).max() < LNL_ATOL
    # the window starts span (nearly) the whole admissible range [0, T_ext - 1 - N_t]
    x0 = []
    for n in range(th.shape[1]):
        nv = np.array([math.cos(th[1, n]) * math.cos(point.gmst - th[0, n]),
                       -math.cos(th[1, n]) * math.sin(point.gmst - th[0, n]), math.sin(th[1, n])])
        dt = -(point.det_pos @ nv) / C_SI
        x0.append((th[6, n] + dt - point.t_start) * point.fs - point.n_window / 2)
    x0 = np.array(x0)
    assert x0.min() < 8 and x0.max() > point.T_ext - 1 - point.n_window - 8


@pytest.mark.parametrize("prec", PRECS)
def test_no_data_and_no_model_power(ile, orc, prec):
    base = S.workload_point(S.FULL)
    th = S.workload_samples(S.FULL, 700)
    # Q = 0: lnL(j) = -A for every window bin, so lnL_t = -A exactly
    p0 = S.Point(**{**base.__dict__, "Q": np.zeros_like(base.Q)})
    got0 = _ctx(ile, p0, prec).eval(th)
    ref0 = orc.lnL_t(p0, th)
    assert np.abs(got0 - ref0).max() < LNL_ATOL
    assert np.all(ref0 <= 0.0)
    # U = V = 0: the data term alone
    p1 = S.Point(**{**base.__dict__, "U": np.zeros_like(base.U), "V": np.zeros_like(base.V)})
    got1 = _ctx(ile, p1, prec).eval(th)
    ref1 = orc.lnL_t(p1, th)
    assert np.abs(got1 - ref1).max() < LNL_ATOL
    # and the two parts add up to the full likelihood inside each window bin (checked through the
    # grid of a few samples: lnL(j) = data(j) - A)
    ctx = _ctx(ile, base, prec)
    full = ctx.eval(th[:, :5], grid=True)
    data = _ctx(ile, p1, prec).eval(th[:, :5], grid=True)
    np.testing.assert_allclose(full - data, np.repeat(got0[:5, None], full.shape[1], axis=1), atol=2 * LNL_ATOL)


def test_largest_launch(ile, orc):
    """2^23 samples in one call (the largest adaptive iteration): every value finite, a random
    subset within tolerance of the oracle."""
    point = S.workload_point(S.FULL)
    N = 1 << 23
    th = S.prior_samples(np.random.default_rng(2026), N)
    got = _ctx(ile, point, "bf16x3").eval(th)
    assert got.shape == (N,) and np.all(np.isfinite(got))
    idx = np.random.default_rng(7).choice(N, 512, replace=False)
    assert np.abs(got[idx] - orc.lnL_t(point, th[:, idx])).max() < LNL_ATOL


def test_largest_adaptive_iteration(ile, orc):
    """n_per_iter = 2^23: the device sampler's last 4096 draws are the oracle's, bit for bit in
    the bins; the iteration's estimate is finite and its sample count exact."""
    point = S.workload_point(S.FULL)
    N = 1 << 23
    lo, hi = ile.default_ranges()
    cfg = ile.make_adapt_cfg(seed=0x5EED, n_per_iter=N, adapt_mask=0b11, point_id=9)
    ctx = _ctx(ile, point, "bf16x3")
    res = ctx.adapt_run(cfg)
    assert res["n_total"] == N and math.isfinite(res["ln_L"])
    theta, lwp, bins, lnl = ctx.adapt_last()
    smp = orc.make_sampler(lo, hi, [1, 1, 0, 0, 0, 0, 0], np.stack([orc.cdf_uniform() for _ in range(7)]))
    n0 = N - 4096
    rt, rl, rb = orc.sample(smp, 0x5EED, 0, 9, n0, 4096)
    np.testing.assert_array_equal(bins[:, n0:], rb)
    np.testing.assert_allclose(theta[6, n0:], rt[6], atol=1e-9)
    assert np.abs(lwp[n0:] - rl).max() < 1e-4
    assert np.abs(lnl[n0:n0 + 256] - orc.lnL_t(point, theta[:, n0:n0 + 256])).max() < LNL_ATOL
