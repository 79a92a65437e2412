"""GPU adjoint (ile_eval_grad / ile_integrate_grad and the autograd wrappers) against the FP64
oracle's analytic gradient and FP64 central differences (needs a GB300).

Bar: every gradient component within GRAD_RTOL of the oracle, relative to the size of that
component (|g| plus its RMS over the compared set), in FP32 arithmetic with FP64 sums over
samples.  Why 1e-3: the backward contractions sum N_t = 512 products per (sample, row) and the
window softmax is recomputed from an FP32 forward whose lnL is within ~1e-4 of the oracle, so the
relative error of a component is ~1e-4 at worst; 1e-3 leaves a 10x margin.
The interpolation slope (d/d ra, d/d dec, d/d t_c) jumps where the window start crosses a bin
edge; the device decides the bin in FP32, the oracle in FP64, so samples whose fractional start
lies within KINK of an edge are left out of those three components (about 1% of samples).
"""
import math

import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-3
LNL_ATOL = 1e-3
LNMARG_ATOL = 1e-4
KINK = 1e-3


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


def _near_kink(orc, point, th):
    """True for samples whose window start in some detector lies within KINK of a bin edge."""
    out = np.zeros(th.shape[1], bool)
    for n in range(th.shape[1]):
        for k in range(point.det_pos.shape[0]):
            dt = orc.delay(point.det_pos[k], th[0, n], th[1, n], point.gmst)
            x = (th[6, n] - 0.5 * point.n_window / point.fs + dt - point.t_start) * point.fs
            f = x - math.floor(x)
            out[n] |= (f < KINK) or (f > 1 - KINK)
    return out


def _assert_close(got, ref, what, rtol=GRAD_RTOL):
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    scale = np.sqrt(np.mean(ref ** 2)) if ref.size else 0.0
    err = np.abs(got - ref)
    bound = rtol * (np.abs(ref) + scale) + 1e-12
    worst = np.argmax(err / bound)
    assert np.all(err <= bound), (what, np.unravel_index(worst, ref.shape), got.flat[worst], ref.flat[worst])


def _check_theta(orc, point, th, got, ref):
    kink = _near_kink(orc, point, th)
    for d in range(7):
        sel = ~kink if d in (0, 1, 6) else np.ones(th.shape[1], bool)
        _assert_close(got[d, sel], ref[d, sel], f"theta[{d}]")
    assert kink.mean() < 0.05


def _compare_all(ile, orc, point, th, g, prec="fp32"):
    ctx = _ctx(ile, point, prec)
    out = ctx.eval_grad(th, g, want_lnL=True)
    lnl, gth, gQ, gU, gV = orc.lnL_t_grad(point, th, g)
    assert np.abs(out["lnL"] - lnl).max() < LNL_ATOL
    _check_theta(orc, point, th, out["theta"], gth)
    _assert_close(out["Q"], gQ, "Q")
    _assert_close(out["U"], gU, "U")
    _assert_close(out["V"], gV, "V")
    return out


# fp32 contexts recompute D(n, j) and contract on CUDA cores; bf16x3 contexts take the window
# softmax from the fused tensor-core forward kernel and, where 64 samples' rows fit shared memory
# (N_t <= 512), run the E / slope contraction on the tensor cores as well
PRECS = ["fp32", "bf16x3"]


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("n_window", [512, 1024])
def test_grad_repeatable_and_output_subsets_equal_full_call(ile, prec, n_window):
    """The gradient call gives the same bits on every run (dQ sums over samples in the delay
    sort's order, which keeps equal keys in the caller's order), and a call that asks for some of
    the outputs returns them bit for bit as the call that asks for all of them.  700 samples over
    3 detectors: several 32-sample dQ chunks and sort buckets holding more than one sample."""
    point = S.make_point(S.SEED_BASE + 61, 3, 9, n_window, spectrum="decay")
    th = S.workload_samples(S.GRAD, 700)
    g = np.random.default_rng(8).normal(size=th.shape[1])
    ctx = _ctx(ile, point, prec)
    full = ctx.eval_grad(th, g, want_lnL=True)
    for _ in range(3):
        again = ctx.eval_grad(th, g, want_lnL=True)
        for key in full:
            assert np.array_equal(again[key], full[key]), key
    for want, lnl in [(("Q",), False), ((), True), (("theta",), False), (("U", "V"), False), (("Q",), True)]:
        part = ctx.eval_grad(th, g, want=want, want_lnL=lnl)
        for key in list(want) + (["lnL"] if lnl else []):
            assert np.array_equal(part[key], full[key]), (want, lnl, key)


@pytest.mark.parametrize("prec", PRECS)
def test_grad_adjoint_K3_M21_Nt512(ile, orc, prec):
    """Three detectors, 21 modes, 512-bin window (the adjoint workload's geometry), 2^10 samples."""
    point = S.workload_point(S.GRAD)
    th = S.workload_samples(S.GRAD, 1024)
    g = np.random.default_rng(7).normal(size=th.shape[1])
    _compare_all(ile, orc, point, th, g, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_grad_two_detectors_ragged(ile, orc, prec):
    """K = 2, M = 2, N_t = 256; 300 samples = 4 tiles of 64 and a ragged tail."""
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 300)
    g = np.random.default_rng(8).uniform(0.5, 1.5, th.shape[1])
    _compare_all(ile, orc, point, th, g, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_grad_four_detectors_nt512(ile, orc, prec):
    """K = 4 (H1/L1/V1/K1), M = 9, N_t = 512: four detectors through the 64-sample tensor-core
    contraction of bf16x3 contexts; 333 samples (a ragged last CTA)."""
    point = S.make_point(S.SEED_BASE + 63, 4, 9, 512, spectrum="decay")
    th = S.prior_samples(np.random.default_rng(64), 333)
    g = np.random.default_rng(65).normal(size=th.shape[1])
    _compare_all(ile, orc, point, th, g, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_grad_long_window_four_detectors(ile, orc, prec):
    """N_t = 1024 (32-sample tiles; the bf16x3 context keeps the CUDA-core contraction), K = 4, M = 9."""
    point = S.make_point(S.SEED_BASE + 60, 4, 9, 1024, spectrum="decay")
    th = S.prior_samples(np.random.default_rng(61), 200)
    g = np.random.default_rng(62).normal(size=th.shape[1])
    _compare_all(ile, orc, point, th, g, prec)


def test_grad_matches_fp64_central_differences(ile, orc):
    """GPU gradient vs central differences (step 1e-6) of the FP64 oracle lnL_t."""
    point = S.workload_point(S.GRAD)
    th = S.workload_samples(S.GRAD, 48)
    got = _ctx(ile, point).eval_grad(th, want=("theta",))["theta"]
    kink = _near_kink(orc, point, th)
    steps = np.array([1e-6, 1e-6, 1e-6, 1e-6, 1e-6, 1e-6, 1e-6])
    fd = np.zeros_like(got)
    for n in range(th.shape[1]):
        for d in range(7):
            h = steps[d] * (th[5, n] if d == 5 else 1.0)
            if d == 6:
                h = 1e-8  # seconds: 4e-5 bins, well inside one interpolation bin
            tp, tm = th[:, n].copy(), th[:, n].copy()
            tp[d] += h
            tm[d] -= h
            fd[d, n] = (orc.lnL_t(point, tp[:, None])[0] - orc.lnL_t(point, tm[:, None])[0]) / (2 * h)
    _check_theta(orc, point, th[:, ~kink], got[:, ~kink], fd[:, ~kink])


@pytest.mark.parametrize("prec", PRECS)
def test_grad_full_size_sampled(ile, orc, prec):
    """2^18 samples through the full launch; the upstream weights are non-zero on 192 random
    samples only, so the oracle can check g_theta on those and the Q/U/V sums exactly."""
    point = S.workload_point(S.GRAD)
    th = S.workload_samples(S.GRAD)
    N = th.shape[1]
    rng = np.random.default_rng(9)
    idx = np.sort(rng.choice(N, 192, replace=False))
    g = np.zeros(N)
    g[idx] = rng.normal(size=idx.size)
    out = _ctx(ile, point, prec).eval_grad(th, g)
    rest = np.ones(N, bool)
    rest[idx] = False
    assert np.all(out["theta"][:, rest] == 0.0)
    _, gth, gQ, gU, gV = orc.lnL_t_grad(point, th[:, idx], g[idx])
    _check_theta(orc, point, th[:, idx], out["theta"][:, idx], gth)
    _assert_close(out["Q"], gQ, "Q")
    _assert_close(out["U"], gU, "U")
    _assert_close(out["V"], gV, "V")


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_integrate_grad_matches_oracle(ile, orc, prec):
    """d ln L_marg / d(theta, Q, U, V) = oracle gradient with weights w_n / sum w."""
    point = S.workload_point(S.GRAD)
    th = S.workload_samples(S.GRAD, 2048)
    rng = np.random.default_rng(10)
    lp = rng.normal(0.0, 0.3, th.shape[1])
    lps = rng.normal(0.0, 0.3, th.shape[1])
    res, out = _ctx(ile, point, prec).integrate_grad(th, lp, lps)
    lnl = orc.lnL_t(point, th)
    st = orc.mc_stats(lnl + lp - lps)
    assert abs(res["ln_L"] - st["ln_I"]) < LNMARG_ATOL
    lnw = lnl + lp - lps
    w = np.exp(lnw - lnw.max())
    w /= w.sum()
    _, gth, gQ, gU, gV = orc.lnL_t_grad(point, th, w)
    _check_theta(orc, point, th, out["theta"], gth)
    _assert_close(out["Q"], gQ, "Q")
    _assert_close(out["U"], gU, "U")
    _assert_close(out["V"], gV, "V")


def _torch_leaves(torch, point, dev):
    Q = torch.tensor(np.stack([point.Q.real, point.Q.imag], -1), dtype=torch.float64, device=dev, requires_grad=True)
    U = torch.tensor(np.stack([point.U.real, point.U.imag], -1), dtype=torch.float64, device=dev, requires_grad=True)
    V = torch.tensor(np.stack([point.V.real, point.V.imag], -1), dtype=torch.float64, device=dev, requires_grad=True)
    return Q, U, V


def test_autograd_lnLt(ile, orc):
    import torch
    from paper_2210_07912_gb300 import autograd as A
    point = S.workload_point(S.GRAD)
    th = S.workload_samples(S.GRAD, 512)
    ctx = _ctx(ile, point)
    dev = torch.device("cuda:0")
    x = torch.tensor(th, dtype=torch.float64, device=dev, requires_grad=True)
    Q, U, V = _torch_leaves(torch, point, dev)
    g = np.random.default_rng(11).normal(size=th.shape[1])
    y = A.lnL_t(ctx, x, Q, U, V)
    assert np.abs(y.detach().cpu().numpy() - orc.lnL_t(point, th)).max() < LNL_ATOL
    (y * torch.tensor(g, device=dev)).sum().backward()
    ref = ctx.eval_grad(th, g)
    # per-sample gradients are bit-identical; the Q sums follow the delay-sorted sample order,
    # whose order inside one delay bucket is not unique, so they agree to FP32 summation order
    np.testing.assert_array_equal(x.grad.cpu().numpy(), ref["theta"])
    for name, t in (("Q", Q), ("U", U), ("V", V)):
        r = ref[name]
        np.testing.assert_allclose(t.grad.cpu().numpy(), r, rtol=1e-5, atol=1e-6 * np.abs(r).max(), err_msg=name)


def test_autograd_lnLmarg(ile, orc):
    import torch
    from paper_2210_07912_gb300 import autograd as A
    point = S.workload_point(S.GRAD)
    th = S.workload_samples(S.GRAD, 1024)
    ctx = _ctx(ile, point)
    dev = torch.device("cuda:0")
    x = torch.tensor(th, dtype=torch.float64, device=dev, requires_grad=True)
    Q, U, V = _torch_leaves(torch, point, dev)
    L = A.lnL_marg(ctx, x, None, None, Q, U, V)
    (2.5 * L).backward()
    lnl = orc.lnL_t(point, th)
    assert abs(L.item() - orc.mc_stats(lnl)["ln_I"]) < LNMARG_ATOL
    w = np.exp(lnl - lnl.max())
    w = 2.5 * w / w.sum()
    _, gth, gQ, gU, gV = orc.lnL_t_grad(point, th, w)
    _check_theta(orc, point, th, x.grad.cpu().numpy(), gth)
    _assert_close(Q.grad.cpu().numpy(), gQ, "Q")
    _assert_close(U.grad.cpu().numpy(), gU, "U")
    _assert_close(V.grad.cpu().numpy(), gV, "V")


def test_grad_errors(ile):
    point = S.workload_point(S.SMALL)
    c = ile.Context(0, None, "fp32")
    th = S.workload_samples(S.SMALL, 8)
    with pytest.raises(ile.IleError) as e:
        c.eval_grad(th)
    assert e.value.status == ile.ILE_E_STATE
    c.set_data(point)
    assert c.eval_grad(th[:, :0], want=("theta",))["theta"].shape == (7, 0)
    lib = ile.load()
    st = lib.ile_eval_grad(c._h, ile._np_ptr(np.ascontiguousarray(th)), 8, ile._np_ptr(np.ones(8)), None, None,
                           None, None, None, 0)
    assert st == ile.ILE_E_ARG
    bad = th.copy()
    bad[6, 3] = 0.05  # t_c far outside the window
    with pytest.raises(ile.IleError) as e:
        c.eval_grad(bad)
    assert e.value.status == ile.ILE_E_RANGE
    # the context stays usable
    assert np.all(np.isfinite(c.eval_grad(th)["theta"]))
