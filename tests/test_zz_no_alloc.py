"""The allocation-free Monte Carlo reduction, ile_mc_reduce_noalloc, against ile_integrate.

Some callers cannot allocate device memory (a host framework's memory pool, a graph-capture
region, a pre-sized service); for them the library offers one reduction whose scratch is a fixed
array inside the library.  The file name sorts last so that a `-x` run reaches every other test
before this one; the tests here do not depend on that order (they also pass alone in a fresh
process, where the entry point's first call is the first use of the library's device code)."""
import ctypes

import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
LNMARG_ATOL = 1e-4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_07912_gb300 import ile
    ile.load()
    return torch, ile


def test_noalloc_reduction_matches_integrate_twice(env):
    torch, ile = env
    point = S.workload_point(S.SMALL)
    ctx = ile.Context(0, None, "fp32")
    ctx.set_data(point)
    lib = ile.load()
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    for call, (N, seed) in enumerate([(12345, 1), (1 << 15, 2)]):  # two calls in a row, different sizes
        th = S.prior_samples(np.random.default_rng(seed), N)
        rng = np.random.default_rng(seed + 10)
        d_th = torch.from_numpy(th).cuda()
        d_lp = torch.from_numpy(rng.normal(0, 0.3, N)).cuda()
        d_lps = torch.from_numpy(rng.normal(0, 0.3, N)).cuda()
        d_lnl = torch.empty(N, dtype=torch.float64, device="cuda")
        ref = torch.empty(8, dtype=torch.float64, device="cuda")
        got = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ctx.integrate_device(d_th, ref, ln_prior=d_lp, ln_ps=d_lps, lnL_out=d_lnl)  # existing entry point
        ctx.sync()
        st = lib.ile_mc_reduce_noalloc(ctypes.c_void_p(d_lnl.data_ptr()), ctypes.c_void_p(d_lp.data_ptr()),
                                       ctypes.c_void_p(d_lps.data_ptr()), N, ctypes.c_void_p(got.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream))
        assert st == ile.ILE_OK, (call, st)
        stream.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert abs(g[0] - r[0]) < LNMARG_ATOL, (call, g[0], r[0])
        np.testing.assert_allclose(g[1:7], r[1:7], rtol=1e-12, atol=1e-300)
    # the python wrapper (default stream) gives the same numbers
    got2 = torch.empty(8, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ile.mc_reduce_noalloc(d_lnl, got2, ln_prior=d_lp, ln_ps=d_lps)
    torch.cuda.synchronize()
    assert abs(got2[0].item() - ref[0].item()) < LNMARG_ATOL


def test_noalloc_rejects_oversize_and_bad_arguments(env):
    torch, ile = env
    lib = ile.load()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.ile_mc_reduce_noalloc(ctypes.c_void_p(x.data_ptr()), None, None, ile.NOALLOC_MAX_SAMPLES + 1,
                                   ctypes.c_void_p(x.data_ptr()), None)
    assert st == ile.ILE_E_ARG
    assert lib.ile_mc_reduce_noalloc(None, None, None, 4, ctypes.c_void_p(x.data_ptr()), None) == ile.ILE_E_ARG
    assert lib.ile_mc_reduce_noalloc(ctypes.c_void_p(x.data_ptr()), None, None, 0,
                                     ctypes.c_void_p(x.data_ptr()), None) == ile.ILE_E_ARG


def test_noalloc_at_the_scratch_limit_against_the_oracle(env):
    """N = ILE_NOALLOC_MAX_SAMPLES fills every partial slot of the fixed array; the result must
    equal the oracle's FP64 Monte Carlo sums of Eq. (eq:lnL:MonteCarlo) on the same ln w values."""
    torch, ile = env
    import oracle
    N = ile.NOALLOC_MAX_SAMPLES
    rng = np.random.default_rng(77)
    lnl = rng.normal(-3.0, 2.0, N)
    lp = rng.normal(0.0, 0.5, N)
    lps = rng.normal(0.0, 0.5, N)
    ref = oracle.mc_stats(lnl + lp - lps)
    d = [torch.from_numpy(a).cuda() for a in (lnl, lp, lps)]
    for _ in range(2):  # two calls in a row share the array
        got = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ile.mc_reduce_noalloc(d[0], got, ln_prior=d[1], ln_ps=d[2])
        torch.cuda.synchronize()
        g = got.cpu().numpy()
        assert abs(g[0] - ref["ln_I"]) < LNMARG_ATOL, (g[0], ref["ln_I"])
        assert g[4] == ref["m"]
        np.testing.assert_allclose([g[1], g[2], g[3], g[5], g[6]],
                                   [ref["sigma_ln"], ref["n_eff"], ref["ess"], ref["s1"], ref["s2"]], rtol=1e-10)


def test_noalloc_wrapper_rejects_wrong_dtype_and_short_tensors(env):
    torch, ile = env
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    res = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ile.IleError):
        ile.mc_reduce_noalloc(x.float(), res)
    with pytest.raises(ile.IleError):
        ile.mc_reduce_noalloc(x, res, ln_prior=torch.zeros(4, dtype=torch.float64, device="cuda"))
    with pytest.raises(ile.IleError):
        ile.mc_reduce_noalloc(x, torch.zeros(4, dtype=torch.float64, device="cuda"))
