"""GPU-vs-oracle parity of the correlated sky-pair mixture (Sec. "Adaptive sampling with gaussian
mixture models": correlated sampling in a subset of dimensions; App. "Gaussian mixture model
implementation"), through the C ABI.

The component of every sample is an integer decision and agrees bit for bit with the oracle given
the same mixture.  The accepted point follows from FP32 (device) or FP64 (oracle) arithmetic; a
candidate that lands within rounding of the rectangle's edge can be kept by one side and rejected
by the other, after which that sample's draws differ (both are valid draws of the same
distribution): the tests require such samples to be rare and compare every other sample's values
at FP32 resolution.  The EM + merge update is compared on the device's own samples and weights."""
import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

PAIR = dict(w=[0.5, 0.3, 0.2], mu=[[1.2, 0.4], [4.0, -0.5], [5.6, 0.7]],
            cov=[[0.3, 0.12, 0.08], [0.8, -0.3, 0.2], [0.2, 0.05, 0.05]])


@pytest.fixture(scope="module")
def ile():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_07912_gb300 import ile as I
    I.load()
    return I


def _resume_with_pair(ile, pair, n_iter, n=4000.0):
    r = ile.AdaptResult()
    r.n_iter = n_iter
    r.max_lnw = -np.inf
    for d in range(7):
        for b in range(101):
            r.cdf[d][b] = (b << 32) // 100
    C = len(pair["w"])
    r.gmm_pair_components = C
    for c in range(C):
        r.gmm_pair_w[c] = pair["w"][c]
        for j in range(2):
            r.gmm_pair_mu[c][j] = pair["mu"][c][j]
        for j in range(3):
            r.gmm_pair_cov[c][j] = pair["cov"][c][j]
    r.gmm_pair_n = n
    return r


def _orc_pair(pair, n):
    return dict(w=np.array(pair["w"], float), mu=np.array(pair["mu"], float), cov=np.array(pair["cov"], float), n=n)


def test_pair_sampler_and_update_match_oracle(ile, orc):
    point = S.workload_point(S.SMALL)
    ctx = ile.Context(0, None, "fp32")
    ctx.set_data(point)
    lo, hi = ile.default_ranges()
    N, seed, pid, it0 = 16384, 0x5EED5, 3, 4
    cfg = ile.make_adapt_cfg(seed=seed, n_per_iter=N, adapt_mask=0b11, point_id=pid, gmm_pair=True,
                             gmm_components=3, gmm_em_iters=5)
    ctx.adapt_init(cfg, _resume_with_pair(ile, PAIR, it0))
    ctx.adapt_step(1)
    theta, lwp, comp, lnl = ctx.adapt_last()
    res = ctx.adapt_get()

    model = _orc_pair(PAIR, 4000.0)
    cdf = np.stack([orc.cdf_uniform() for _ in range(7)])
    smp = orc.make_sampler(lo, hi, [1, 1, 0, 0, 0, 0, 0], cdf, None, point.gmst, None, model)
    rt, rl, rb, ru = orc.sample(smp, seed, it0, pid, 0, N, with_u=True)
    np.testing.assert_array_equal(comp[0], rb[0])  # the components: bit-exact
    np.testing.assert_array_equal(comp[1], comp[0])
    u0, u1 = theta[0], np.sin(theta[1])
    same = (np.abs(u0 - ru[0]) < 1e-4) & (np.abs(u1 - ru[1]) < 1e-4)
    assert same.mean() > 0.999, same.mean()  # only edge acceptances may differ
    assert np.abs(u0 - ru[0])[same].max() < 2e-5 and np.abs(u1 - ru[1])[same].max() < 2e-5
    assert np.abs(lwp - rl)[same].max() < 2e-4
    assert np.all((u0 >= lo[0]) & (u0 <= hi[0]) & (u1 >= lo[1]) & (u1 <= hi[1]))
    # ln p - ln p_s of every device sample against the oracle's density at the device's point
    Z = orc.gmm2_masses(model, lo[:2], hi[:2])
    for n in range(0, N, 611):
        want = -np.log(hi[0] - lo[0]) - np.log(hi[1] - lo[1]) - orc.gmm2_lnpdf(model, lo[:2], hi[:2], [u0[n], u1[n]], Z)
        assert abs(lwp[n] - want) < 2e-4, n
    # the update: EM from the resumed mixture and the merge, on the device's samples and weights
    lnw = lnl + lwp
    w = np.exp(lnw - lnw.max())
    ref = orc.gmm2_update(model, u0, u1, w, 5, lo[:2], hi[:2])
    got = res["pair"]
    assert got["n"] == ref["n"] == 4000.0 + N
    np.testing.assert_allclose(got["mu"], ref["mu"], atol=1e-4)
    np.testing.assert_allclose(got["cov"], ref["cov"], rtol=1e-3, atol=1e-6)
    np.testing.assert_allclose(got["w"], ref["w"], atol=1e-5)
    assert res["gmm"][0] is None and res["gmm"][1] is None


def test_pair_adaptive_run_matches_oracle_and_resumes(ile, orc):
    """From the initial mixture both sides draw the same first iteration (ln L within 1e-4); the
    run concentrates the pair; a run resumed from its checkpoint continues bit for bit."""
    point = S.workload_point(S.SMALL)
    lo, hi = ile.default_ranges()
    N = 8192
    cfg = ile.make_adapt_cfg(seed=77, n_per_iter=N, n_iter=3, adapt_mask=0b11, point_id=1, gmm_pair=True,
                             gmm_components=3, gmm_em_iters=4)
    ctx = ile.Context(0, None, "bf16x3")
    ctx.set_data(point)
    res = ctx.adapt_run(cfg)
    ref = orc.adapt_run(point, 77, N, 3, 0b11, 0.1, lo, hi, point_id=1, gmm_pair=True, gmm_components=3,
                        gmm_em_iters=4)
    assert abs(res["iter_ln_L"][0] - ref["iters"][0]["ln_I"]) < 1e-4
    for i in range(3):
        assert abs(res["iter_ln_L"][i] - ref["iters"][i]["ln_I"]) < 5e-3
    np.testing.assert_allclose(res["pair"]["mu"], ref["pair"]["mu"], atol=5e-3)
    # checkpoint after one iteration, resume for two more: the same as three in a row
    cfg1 = ile.make_adapt_cfg(seed=77, n_per_iter=N, n_iter=1, adapt_mask=0b11, point_id=1, gmm_pair=True,
                              gmm_components=3, gmm_em_iters=4)
    ctx.adapt_init(cfg1)
    ctx.adapt_step(1)
    chk = ctx.adapt_get(raw=True)
    ctx.adapt_init(cfg1, chk)
    ctx.adapt_step(2)
    resumed = ctx.adapt_get()
    assert resumed["ln_L"] == res["ln_L"]
    np.testing.assert_array_equal(resumed["pair"]["cov"], res["pair"]["cov"])


def test_pair_in_rotated_frame_and_errors(ile, orc):
    point = S.workload_point(S.FULL)
    _, pos = S.detector_arrays(3)
    cfg = ile.make_adapt_cfg(seed=9, n_per_iter=1 << 14, n_iter=2, adapt_mask=0b11, point_id=0, gmm_pair=True,
                             gmm_components=4, gmm_em_iters=3, sky_pole=pos[1] - pos[0])
    ctx = ile.Context(0, None, "bf16x3")
    ctx.set_data(point)
    r = ctx.adapt_run(cfg)
    assert np.isfinite(r["ln_L"]) and r["pair"] is not None and len(r["pair"]["w"]) == 4
    theta, _, _, lnl = ctx.adapt_last()
    assert np.abs(lnl[:1000] - orc.lnL_t(point, theta[:, :1000])).max() < 1e-3
    # the pair needs both sky variables adaptive and outside the separable mixtures
    bad = ile.make_adapt_cfg(seed=9, n_per_iter=1024, adapt_mask=0b01, gmm_pair=True)
    with pytest.raises(ile.IleError):
        ctx.adapt_init(bad)
    bad2 = ile.make_adapt_cfg(seed=9, n_per_iter=1024, adapt_mask=0b11, gmm_mask=0b10, gmm_pair=True)
    with pytest.raises(ile.IleError):
        ctx.adapt_init(bad2)
