"""GPU-vs-oracle parity of the device sampler (S0) and the adaptive Monte Carlo integrator (S6),
through the C ABI.  Integer decisions (histogram bins, integer cumulative tables) must agree bit
for bit; floating-point values within the tolerances of the path (lnL 1e-3, ln L_marg 1e-4)."""
import math

import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ile():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_07912_gb300 import ile as I
    I.load()
    return I


def _ranges(ile):
    return ile.default_ranges()


def _random_tables(orc, seed):
    rng = np.random.default_rng(seed)
    return np.stack([orc.cdf_from_hist(rng.gamma(0.4, size=100), 0.1) for _ in range(7)])


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_sampler_bits_and_values_match_oracle(ile, orc, prec):
    point = S.workload_point(S.SMALL)
    ctx = ile.Context(0, None, prec)
    ctx.set_data(point)
    lo, hi = _ranges(ile)
    mask = 0b1111011  # every dimension but psi adaptive
    cfg = ile.make_adapt_cfg(seed=0xC0FFEE12345, n_per_iter=20000, adapt_mask=mask, point_id=7)
    tables = _random_tables(orc, 5)
    resume = ile.AdaptResult()
    resume.n_iter = 3
    resume.max_lnw = -np.inf
    np.ctypeslib.as_array(resume.cdf)[:] = tables
    ctx.adapt_init(cfg, resume)
    ctx.adapt_step(1)
    theta, lwp, bins, lnl = ctx.adapt_last()
    smp = orc.make_sampler(lo, hi, [(mask >> d) & 1 for d in range(7)], tables)
    rt, rl, rb = orc.sample(smp, 0xC0FFEE12345, 3, 7, 0, 20000)
    np.testing.assert_array_equal(bins, rb)  # integer decisions: bit-exact
    np.testing.assert_allclose(theta[[0, 2, 4]], rt[[0, 2, 4]], atol=2e-6)
    # dec and iota: their sampling variables sin(dec) and cos(iota) at FP32 resolution everywhere,
    # and the angles themselves to 2e-6 rad away from the poles (asin / acos amplify an FP32
    # rounding of the sampling variable by 1 / sqrt(1 - u^2) there)
    for d, f in ((1, np.sin), (3, np.cos)):
        u_gpu, u_ref = f(theta[d]), f(rt[d])
        np.testing.assert_allclose(u_gpu, u_ref, atol=3e-7)
        away = np.abs(u_ref) < 0.99
        assert away.sum() > 0.9 * away.size
        np.testing.assert_allclose(theta[d][away], rt[d][away], atol=2e-6)
    np.testing.assert_allclose(theta[6], rt[6], atol=1e-9)
    np.testing.assert_allclose(theta[5], rt[5], rtol=2e-6)
    assert np.abs(lwp - rl).max() < 1e-4
    # the likelihood of the drawn samples matches the oracle on the same (device) samples
    ref = orc.lnL_t(point, theta[:, :3000])
    assert np.abs(lnl[:3000] - ref).max() < 1e-3


def test_histograms_and_tables_match_oracle(ile, orc):
    point = S.workload_point(S.SMALL)
    ctx = ile.Context(0, None, "fp32")
    ctx.set_data(point)
    mask = 0b0101011
    cfg = ile.make_adapt_cfg(seed=99, n_per_iter=30000, adapt_mask=mask, eps=0.05)
    ctx.adapt_init(cfg)
    ctx.adapt_step(1)
    res = ctx.adapt_get()
    theta, lwp, bins, lnl = ctx.adapt_last()
    lnw = lnl + lwp
    for d in range(7):
        if not (mask >> d) & 1:
            continue
        h = res["hist"][d]
        ref = orc.hist(lnw, bins[d])  # normalised, FP64, from the device's weights and bins
        np.testing.assert_allclose(h / h.sum(), ref, rtol=2e-5, atol=1e-9)
        # next table: bit-exact function of the device histogram
        np.testing.assert_array_equal(res["cdf"][d], orc.cdf_from_hist(h, 0.05))
    # fixed dimensions keep their uniform table
    for d in (2, 4, 6):
        np.testing.assert_array_equal(res["cdf"][d], orc.cdf_uniform())


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
def test_first_iteration_matches_independent_oracle_run(ile, orc, prec):
    """Iteration 0 (uniform tables): the oracle draws the same samples itself (same Philox words)
    and evaluates them in FP64; ln L estimates agree within 1e-4."""
    point = S.workload_point(S.SMALL)
    ctx = ile.Context(0, None, prec)
    ctx.set_data(point)
    lo, hi = _ranges(ile)
    N = 16384
    cfg = ile.make_adapt_cfg(seed=2024, n_per_iter=N, adapt_mask=0b11, point_id=1)
    res = ctx.adapt_run(cfg)
    ref = orc.adapt_run(point, 2024, N, 1, 0b11, 0.1, lo, hi, point_id=1)
    assert abs(res["iter_ln_L"][0] - ref["iters"][0]["ln_I"]) < 1e-4
    assert abs(res["ln_L"] - ref["pooled"]["ln_I"]) < 1e-4
    assert abs(res["n_eff"] - ref["pooled"]["n_eff"]) < 1e-3 * ref["pooled"]["n_eff"]


def test_adaptive_run_matches_oracle_run(ile, orc):
    """Five adaptive iterations on both sides from the same seed.  The tables are refit from
    weights that differ at the 1e-6 level, so the sample sets can differ in a few samples per
    iteration; the pooled estimates must agree within their Monte Carlo errors, and in practice
    agree far closer."""
    point = S.workload_point(S.SMALL)
    ctx = ile.Context(0, None, "fp32")
    ctx.set_data(point)
    lo, hi = _ranges(ile)
    N = 8192
    cfg = ile.make_adapt_cfg(seed=77, n_per_iter=N, n_iter=5, adapt_mask=0b11, point_id=3)
    res = ctx.adapt_run(cfg)
    ref = orc.adapt_run(point, 77, N, 5, 0b11, 0.1, lo, hi, point_id=3)
    sig = math.hypot(res["sigma_ln"], ref["pooled"]["sigma_ln"])
    assert abs(res["ln_L"] - ref["pooled"]["ln_I"]) < 4 * sig + 1e-4
    assert res["n_iter"] == 5 and res["n_total"] == 5 * N
    # the adapted tables are close (same histograms up to the 1e-6 weight differences)
    diff = np.abs(res["cdf"].astype(np.int64) - ref["cdf"].astype(np.int64)).max() / 2.0 ** 32
    assert diff < 1e-3


def test_resume_is_bit_reproducible(ile):
    point = S.workload_point(S.SMALL)
    lo, hi = _ranges(ile)
    cfg = ile.make_adapt_cfg(seed=5, n_per_iter=4096, adapt_mask=0b1100011, point_id=2)
    a = ile.Context(0, None, "bf16x3")
    a.set_data(point)
    a.adapt_init(cfg)
    a.adapt_step(4)
    full = a.adapt_get()
    b = ile.Context(0, None, "bf16x3")
    b.set_data(point)
    b.adapt_init(cfg)
    b.adapt_step(2)
    mid = b.adapt_get(raw=True)
    c = ile.Context(0, None, "bf16x3")
    c.set_data(point)
    c.adapt_init(cfg, mid)
    c.adapt_step(2)
    resumed = c.adapt_get()
    np.testing.assert_array_equal(full["cdf"], resumed["cdf"])
    assert full["ln_L"] == resumed["ln_L"] and full["s2"] == resumed["s2"] and resumed["n_iter"] == 4
    np.testing.assert_array_equal(full["iter_ln_L"], resumed["iter_ln_L"])


def test_adapt_argument_errors(ile):
    point = S.workload_point(S.SMALL)
    ctx = ile.Context(0)
    cfg = ile.make_adapt_cfg(seed=1, n_per_iter=100)
    with pytest.raises(ile.IleError) as e:
        ctx.adapt_init(cfg)
    assert e.value.status == ile.ILE_E_STATE
    ctx.set_data(point)
    for bad in (ile.make_adapt_cfg(seed=1, n_per_iter=0), ile.make_adapt_cfg(seed=1, n_per_iter=10, eps=0.0),
                ile.make_adapt_cfg(seed=1, n_per_iter=10, adapt_mask=1 << 7),
                ile.make_adapt_cfg(seed=1, n_per_iter=10, lo=[0, -2, 0, -1, 0, 100, 0], hi=[1, 1, 1, 1, 1, 1000, 1])):
        with pytest.raises(ile.IleError) as e:
            ctx.adapt_init(bad)
        assert e.value.status == ile.ILE_E_ARG
    with pytest.raises(ile.IleError) as e:
        ctx.adapt_step(1)
    assert e.value.status == ile.ILE_E_STATE


def test_rotated_sky_sampler_matches_oracle(ile, orc):
    """Rotated network-frame sky variables (pole along the H1-L1 baseline): identical bins, the
    (ra, dec) the frame maps them to within FP32 rounding, ln p - ln p_s unchanged."""
    point = S.workload_point(S.SMALL)
    ctx = ile.Context(0, None, "bf16x3")
    ctx.set_data(point)
    lo, hi = _ranges(ile)
    _, pos = S.detector_arrays(2)
    pole = pos[1] - pos[0]
    cfg = ile.make_adapt_cfg(seed=4242, n_per_iter=20000, adapt_mask=0b11, point_id=3, sky_pole=pole)
    tables = _random_tables(orc, 6)
    resume = ile.AdaptResult()
    resume.n_iter = 2
    resume.max_lnw = -np.inf
    np.ctypeslib.as_array(resume.cdf)[:] = tables
    ctx.adapt_init(cfg, resume)
    ctx.adapt_step(1)
    theta, lwp, bins, lnl = ctx.adapt_last()
    smp = orc.make_sampler(lo, hi, [1, 1, 0, 0, 0, 0, 0], tables, pole, point.gmst)
    rt, rl, rb = orc.sample(smp, 4242, 2, 3, 0, 20000)
    np.testing.assert_array_equal(bins, rb)
    dra = np.abs(np.angle(np.exp(1j * (theta[0] - rt[0]))))
    assert dra.max() < 1e-4 and np.abs(theta[1] - rt[1]).max() < 1e-4
    assert np.abs(lwp - rl).max() < 1e-4
    ref = orc.lnL_t(point, theta[:, :2000])
    assert np.abs(lnl[:2000] - ref).max() < 1e-3


def test_rotated_sky_adaptive_run_matches_oracle_and_batch(ile, orc):
    point = S.workload_point(S.SMALL)
    lo, hi = _ranges(ile)
    _, pos = S.detector_arrays(2)
    pole = pos[1] - pos[0]
    N = 16384
    cfg = ile.make_adapt_cfg(seed=31, n_per_iter=N, n_iter=1, adapt_mask=0b11, point_id=4, sky_pole=pole)
    ctx = ile.Context(0, None, "bf16x3")
    ctx.set_data(point)
    res = ctx.adapt_run(cfg)
    ref = orc.adapt_run(point, 31, N, 1, 0b11, 0.1, lo, hi, point_id=4, sky_pole=pole)
    assert abs(res["iter_ln_L"][0] - ref["iters"][0]["ln_I"]) < 1e-4
    # the same point in a batch reproduces the single-point run bit for bit
    cfg.n_iter = 3
    single = ctx.adapt_run(cfg)
    b = ile.Batch(0, None, "bf16x3")
    out = b.run([point], [cfg], 3)[0]
    assert out["ln_L"] == single["ln_L"]
    np.testing.assert_array_equal(out["cdf"], single["cdf"])


def test_device_philox_known_answer_vectors(ile):
    """The device sampler's generator reproduces the published Philox4x32-10 known-answer vectors
    (the same vectors pin the oracle's generator in the CPU tests)."""
    import torch
    from test_oracle_pins import philox_kat_vectors
    kat = philox_kat_vectors()
    ck = torch.tensor(np.array([[*c, *k] for c, k, _ in kat], dtype=np.uint32).view(np.int32)).cuda()
    out = torch.zeros((len(kat), 4), dtype=torch.int32, device="cuda")
    ile.philox4x32_10(ck, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    for i, (_, _, want) in enumerate(kat):
        assert [int(x) for x in got[i]] == want, i
