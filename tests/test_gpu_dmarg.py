"""Distance-marginalised likelihood on the GPU (ile_set_distance_marginalization) against the
FP64 oracle (quadrature over D for every window bin), through the C ABI (needs a GB300).
Bar: per-sample and per-bin values within 1e-3 of the oracle, ln L_marg within 1e-4."""
import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "tf32x3", "bf16x3"]
D_MIN, D_MAX = 100.0, 1000.0


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
    c.set_distance_marginalization(True, D_MIN, D_MAX)
    return c


def _scaled(point, g):
    """The same point with every inner product (Q, U, V) scaled by g: a g-times louder network."""
    import dataclasses
    return dataclasses.replace(point, Q=point.Q * g, U=point.U * g, V=point.V * g)


def _loud_point(K=3, M=5, Nt=128, gain=25.0):
    """A point whose quadratic term is ~600x the default (SNR ~ 100): the sharply peaked regime."""
    rng = np.random.default_rng(77)
    amp = rng.normal(0.0, 0.5, K) + 1j * rng.normal(0.0, 0.5, K)
    c_true = gain * amp[:, None] * (rng.normal(size=M) + 1j * rng.normal(size=M))[None, :] * 0.3
    return S.make_point(S.SEED_BASE + 80, K, M, Nt, spectrum="decay", c_true=c_true)


@pytest.mark.parametrize("prec", PRECS)
def test_dmarg_matches_oracle(ile, orc, prec):
    for point, th in ((S.workload_point(S.SMALL), S.workload_samples(S.SMALL, 300)),
                      (S.make_point(S.SEED_BASE + 81, 3, 21, 512, spectrum="decay"), S.workload_samples(S.FULL, 200)),
                      # four detectors with 21 modes: the bf16x3 launch keeps A in shared memory and
                      # has no room for the per-sample interpolant store (it refits every chunk)
                      (S.make_point(S.SEED_BASE + 84, 4, 21, 512, spectrum="decay"), S.workload_samples(S.FULL, 200)),
                      (_loud_point(), S.workload_samples(S.SMALL, 200))):
        got = _ctx(ile, point, prec).eval(th)
        ref = orc.lnL_dmarg(point, th, D_MIN, D_MAX)
        err = np.abs(got - ref).max()
        assert err < 1e-3, (prec, err)


def test_dmarg_per_bin_table_accuracy(ile, orc):
    """Every window bin's ln F(a_j, b) (the ILE_NO_TMARG grid) against the oracle's quadrature:
    exercises the tables over the (a, b) range of a normal point, a loud one and a network 30
    times louder (b up to ~350).  Bar: 1e-3 plus the FP32 precision of the inputs (the data term
    a_j is an FP32 sum, ~2e-6 relative; it only matters once |ln F| >> 100)."""
    for point in (S.workload_point(S.SMALL), _loud_point(), _scaled(S.workload_point(S.SMALL), 30.0)):
        th = S.workload_samples(S.SMALL, 40)
        grid = _ctx(ile, point, "fp32").eval(th, grid=True)
        for n in range(th.shape[1]):
            t = th[:, n].copy()
            t[5] = point.d_ref
            _, data, A = orc.lnL_grid(point, t)
            for j in range(0, point.n_window, 7):
                ref = orc.dmarg_lnF(data[j], A, D_MIN, D_MAX, point.d_ref)
                assert abs(grid[n, j] - ref) < 1e-3 + 2e-6 * abs(ref), (n, j, grid[n, j], ref, data[j], A)


def test_dmarg_tables_over_the_ab_plane(ile, orc):
    """ln F from the tables (ile_dmarg_eval) against the oracle's quadrature on a log-spaced grid
    of b in [1e-5, 1e6] and a in a band around the peak position, both tables and their seam."""
    c = _ctx(ile, S.workload_point(S.SMALL), "fp32")
    rng = np.random.default_rng(90)
    bs = 10.0 ** rng.uniform(-5, 6, 400)
    us = rng.uniform(-0.3, 1.5, 400)  # peak position a / 2b: inside, below and above [0.1, 1]
    a = 2 * bs * us + rng.normal(0, 1, 400) * np.sqrt(bs)
    got = c.dmarg_eval(a, bs)
    ref = np.array([orc.dmarg_lnF(x, y, D_MIN, D_MAX, 100.0) for x, y in zip(a, bs)])
    err = np.abs(got - ref) / (1.0 + 2e-6 * np.abs(ref) / 1e-3)
    i = int(np.argmax(err))
    assert err.max() < 1e-3, (a[i], bs[i], got[i], ref[i])


def test_dmarg_integrate_and_adaptive_run(ile, orc):
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 4096)
    c = _ctx(ile, point, "bf16x3")
    res = c.integrate(th)
    ref = orc.mc_stats(orc.lnL_dmarg(point, th, D_MIN, D_MAX))
    assert abs(res["ln_L"] - ref["ln_I"]) < 1e-4
    # adaptive run: D is not sampled adaptively; the last iteration's likelihoods are the oracle's
    cfg = ile.make_adapt_cfg(seed=5, n_per_iter=8192, n_iter=2, adapt_mask=0b11, point_id=2)
    r = c.adapt_run(cfg)
    assert np.isfinite(r["ln_L"]) and r["n_iter"] == 2
    theta, _, _, lnl = c.adapt_last()
    assert np.abs(lnl[:500] - orc.lnL_dmarg(point, theta[:, :500], D_MIN, D_MAX)).max() < 1e-3


def test_dmarg_switching_and_errors(ile, orc):
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 64)
    c = ile.Context(0, None, "fp32")
    with pytest.raises(ile.IleError) as e:
        c.set_distance_marginalization(True, D_MIN, D_MAX)
    assert e.value.status == ile.ILE_E_STATE
    c.set_data(point)
    with pytest.raises(ile.IleError) as e:
        c.set_distance_marginalization(True, 500.0, 400.0)
    assert e.value.status == ile.ILE_E_ARG
    plain = c.eval(th)
    c.set_distance_marginalization(True, D_MIN, D_MAX)
    with pytest.raises(ile.IleError) as e:
        c.eval_grad(th)
    assert e.value.status == ile.ILE_E_STATE
    assert np.abs(c.eval(th) - orc.lnL_dmarg(point, th, D_MIN, D_MAX)).max() < 1e-3
    c.set_distance_marginalization(False)
    np.testing.assert_allclose(c.eval(th), plain, rtol=0, atol=1e-9)
    c.set_distance_marginalization(True, D_MIN, D_MAX)
    c.set_data(point)  # a new point turns it off
    np.testing.assert_allclose(c.eval(th), plain, rtol=0, atol=1e-9)


@pytest.mark.parametrize("prec", PRECS)
def test_dmarg_ragged_window_and_both_epilogue_paths(ile, orc, prec):
    """A window of 200 bins (three full 64-bin chunks and a ragged chunk of 8), on a quiet point
    (every chunk's data terms within the interpolated range) and on a 25x louder one (most chunks
    wider: per-bin table reads), per sample and per bin against the oracle's quadrature."""
    for gain in (1.0, 25.0):
        point = _scaled(S.make_point(S.SEED_BASE + 83, 3, 9, 200, spectrum="decay"), gain)
        th = S.workload_samples(S.SMALL, 256)
        c = _ctx(ile, point, prec)
        got = c.eval(th)
        ref = orc.lnL_dmarg(point, th, D_MIN, D_MAX)
        assert np.abs(got - ref).max() < 1e-3, (prec, gain, np.abs(got - ref).max())
        grid = c.eval(th[:, :12], grid=True)
        for n in range(12):
            t = th[:, n].copy()
            t[5] = point.d_ref
            _, data, A = orc.lnL_grid(point, t)
            for j in list(range(0, 200, 9)) + [192, 195, 199]:
                want = orc.dmarg_lnF(data[j], A, D_MIN, D_MAX, point.d_ref)
                assert abs(grid[n, j] - want) < 1e-3 + 2e-6 * abs(want), (prec, gain, n, j)
