"""GPU-vs-oracle parity of the Gaussian-mixture sampling prior (Sec. "Adaptive sampling with
gaussian mixture models"; App. "Gaussian mixture model implementation"), through the C ABI.

Component choices are integer decisions and agree bit for bit with the oracle given the same
mixture; sampled values within FP32 rounding; the EM + merge update within the spread that the
FP32 responsibilities and the 1e-3-level lnL differences allow; ln L estimates within 1e-4 on the
first iteration (identical initial mixtures) and within the Monte Carlo error afterwards."""
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


MODELS = {
    1: dict(w=[0.25, 0.5, 0.25], mu=[-0.7, 0.1, 0.8], sigma=[0.1, 0.3, 0.15]),       # sin dec
    3: dict(w=[0.6, 0.399, 1e-3], mu=[-0.95, 0.9, 0.0], sigma=[0.05, 0.2, 0.5]),       # cos iota
    5: dict(w=[0.2, 0.3, 0.5], mu=[150.0, 420.0, 700.0], sigma=[30.0, 80.0, 200.0]),  # distance
}


def _resume_with(ile, models, n_iter, gmm_n=5000.0):
    r = ile.AdaptResult()
    r.n_iter = n_iter
    r.max_lnw = -np.inf
    for d in range(7):
        for b in range(101):
            r.cdf[d][b] = (b << 32) // 100
    for d, m in models.items():
        r.gmm_components[d] = len(m["w"])
        for c in range(len(m["w"])):
            r.gmm_w[d][c], r.gmm_mu[d][c], r.gmm_sigma[d][c] = m["w"][c], m["mu"][c], m["sigma"][c]
        r.gmm_n[d] = gmm_n
    return r


def _oracle_models(models, n):
    out = [None] * 7
    for d, m in models.items():
        out[d] = dict(w=np.array(m["w"], float), mu=np.array(m["mu"], float), sigma=np.array(m["sigma"], float), n=n)
    return out


def test_mixture_sampler_and_update_match_oracle(ile, orc):
    point = S.workload_point(S.SMALL)
    ctx = ile.Context(0, None, "fp32")
    ctx.set_data(point)
    lo, hi = ile.default_ranges()
    N, seed, pid, it0 = 8192, 0xABCDEF, 5, 2
    adapt = 0b0101011  # ra (histogram), sin dec, cos iota, D (mixtures)
    gmask = 0b0101010
    cfg = ile.make_adapt_cfg(seed=seed, n_per_iter=N, adapt_mask=adapt, point_id=pid, gmm_mask=gmask,
                             gmm_components=3, gmm_em_iters=6)
    ctx.adapt_init(cfg, _resume_with(ile, MODELS, it0))
    ctx.adapt_step(1)
    theta, lwp, comp, lnl = ctx.adapt_last()
    res = ctx.adapt_get()

    models = _oracle_models(MODELS, 5000.0)
    cdf = np.stack([orc.cdf_uniform() for _ in range(7)])
    smp = orc.make_sampler(lo, hi, [(adapt >> d) & 1 for d in range(7)], cdf, None, point.gmst, models)
    rt, rl, rb, ru = orc.sample(smp, seed, it0, pid, 0, N, with_u=True)
    np.testing.assert_array_equal(comp, rb)  # component and bin choices: bit-exact
    for d in (1, 3):
        assert np.all(comp[d] < 3)
    np.testing.assert_allclose(theta[5], rt[5], rtol=1e-5)
    assert np.abs(np.sin(theta[1]) - ru[1]).max() < 2e-5
    assert np.abs(np.cos(theta[3]) - ru[3]).max() < 2e-5
    np.testing.assert_allclose(theta[[0, 2, 4, 6]], rt[[0, 2, 4, 6]], atol=2e-6)
    assert np.abs(lwp - rl).max() < 2e-4
    # the update: EM from the resumed mixture on the oracle's own samples and FP64 likelihoods
    lnw = orc.lnL_t(point, rt) + rl
    w = np.exp(lnw - lnw.max())
    for d in (1, 3, 5):
        ref = orc.gmm_update(models[d], ru[d], w, 6, lo[d], hi[d])
        got = res["gmm"][d]
        span = hi[d] - lo[d]
        assert abs(got["n"] - ref["n"]) == 0
        np.testing.assert_allclose(got["mu"], ref["mu"], atol=3e-3 * span)
        np.testing.assert_allclose(got["sigma"], ref["sigma"], rtol=1e-2, atol=1e-4 * span)
        np.testing.assert_allclose(got["w"], ref["w"], atol=3e-3)
        assert abs(got["w"].sum() - 1.0) < 1e-12
    # dimensions without a mixture report none
    assert res["gmm"][0] is None and res["gmm"][2] is None


def test_first_iteration_matches_oracle_and_run_agrees(ile, orc):
    """Iteration 0 starts from the same initial mixtures on both sides (so the same samples);
    later iterations refit from slightly different weights, so they agree within MC errors."""
    point = S.workload_point(S.SMALL)
    lo, hi = ile.default_ranges()
    N = 8192
    cfg = ile.make_adapt_cfg(seed=404, n_per_iter=N, n_iter=4, adapt_mask=0b11, point_id=2, gmm_mask=0b11,
                             gmm_components=4, gmm_em_iters=5)
    ctx = ile.Context(0, None, "bf16x3")
    ctx.set_data(point)
    res = ctx.adapt_run(cfg)
    ref = orc.adapt_run(point, 404, N, 4, 0b11, 0.1, lo, hi, point_id=2, gmm_mask=0b11, gmm_components=4,
                        gmm_em_iters=5)
    assert abs(res["iter_ln_L"][0] - ref["iters"][0]["ln_I"]) < 1e-4
    sig = math.hypot(res["sigma_ln"], ref["pooled"]["sigma_ln"])
    assert abs(res["ln_L"] - ref["pooled"]["ln_I"]) < 4 * sig + 1e-4
    for d in (0, 1):
        g, r = res["gmm"][d], ref["gmm"][d]
        assert g["n"] == r["n"] == 4 * N
        np.testing.assert_allclose(np.sort(g["mu"]), np.sort(r["mu"]), atol=0.05 * (hi[d] - lo[d]))


def test_mixture_and_histogram_estimates_agree(ile):
    """Two unbiased estimators of the same integral: the Gaussian-mixture and the histogram
    sampling priors give ln L_marg within their combined Monte Carlo error."""
    point = S.workload_point(S.SMALL)
    N = 1 << 15
    est = []
    for gmask in (0, 0b0101011):
        cfg = ile.make_adapt_cfg(seed=17, n_per_iter=N, n_iter=8, adapt_mask=0b0101011, point_id=9, gmm_mask=gmask,
                                 gmm_components=3, gmm_em_iters=8)
        ctx = ile.Context(0, None, "bf16x3")
        ctx.set_data(point)
        est.append(ctx.adapt_run(cfg))
    sig = math.hypot(est[0]["sigma_ln"], est[1]["sigma_ln"])
    assert abs(est[0]["ln_L"] - est[1]["ln_L"]) < 4 * sig + 1e-4
    assert est[1]["n_eff"] > 100


def test_mixture_resume_is_bit_reproducible(ile):
    point = S.workload_point(S.SMALL)
    cfg = ile.make_adapt_cfg(seed=8, n_per_iter=4096, adapt_mask=0b0101011, point_id=1, gmm_mask=0b0001010,
                             gmm_components=2, gmm_em_iters=3)
    a = ile.Context(0, None, "bf16x3")
    a.set_data(point)
    a.adapt_init(cfg)
    a.adapt_step(3)
    full = a.adapt_get()
    b = ile.Context(0, None, "bf16x3")
    b.set_data(point)
    b.adapt_init(cfg)
    b.adapt_step(1)
    mid = b.adapt_get(raw=True)
    b.adapt_init(cfg, mid)
    b.adapt_step(2)
    resumed = b.adapt_get()
    assert full["ln_L"] == resumed["ln_L"] and full["s2"] == resumed["s2"]
    for d in (1, 3):
        for k in ("w", "mu", "sigma"):
            np.testing.assert_array_equal(full["gmm"][d][k], resumed["gmm"][d][k])
        assert full["gmm"][d]["n"] == resumed["gmm"][d]["n"] == 3 * 4096
    np.testing.assert_array_equal(full["cdf"], resumed["cdf"])


def test_mixture_argument_errors(ile):
    point = S.workload_point(S.SMALL)
    ctx = ile.Context(0)
    ctx.set_data(point)
    bad = [ile.make_adapt_cfg(seed=1, n_per_iter=64, adapt_mask=0b01, gmm_mask=0b10),
           ile.make_adapt_cfg(seed=1, n_per_iter=64, adapt_mask=0b11, gmm_mask=0b10, gmm_components=0),
           ile.make_adapt_cfg(seed=1, n_per_iter=64, adapt_mask=0b11, gmm_mask=0b10, gmm_components=9),
           ile.make_adapt_cfg(seed=1, n_per_iter=64, adapt_mask=0b11, gmm_mask=0b10, gmm_em_iters=0)]
    for cfg in bad:
        with pytest.raises(ile.IleError) as e:
            ctx.adapt_init(cfg)
        assert e.value.status == ile.ILE_E_ARG
    cfg = ile.make_adapt_cfg(seed=1, n_per_iter=64, adapt_mask=0b1010, gmm_mask=0b1010, gmm_components=3)
    for d, field, val in ((1, "mu", 1.5), (3, "sigma", 0.0), (1, "w", -0.1)):
        r = _resume_with(ile, {1: MODELS[1], 3: MODELS[3]}, 1)
        getattr(r, "gmm_" + field)[d][0] = val
        with pytest.raises(ile.IleError) as e:
            ctx.adapt_init(cfg, r)
        assert e.value.status == ile.ILE_E_ARG
    r = _resume_with(ile, {1: MODELS[1], 3: MODELS[3]}, 1)
    r.gmm_components[3] = 2
    with pytest.raises(ile.IleError) as e:
        ctx.adapt_init(cfg, r)
    assert e.value.status == ile.ILE_E_ARG
    b = ile.Batch(0, None, "bf16x3")
    with pytest.raises(ValueError):
        b.run([point], [cfg], 1)
