"""Pins of the oracle's Gaussian-mixture sampler (Sec. "Adaptive sampling with gaussian mixture
models" and the appendix "Gaussian mixture model implementation"), CPU only.

Each function is tied to something other than itself: the normal quantile to a library and to
Phi(ppf(p)) = p; the truncated-mixture density to quadrature and to scipy's truncnorm; the sampler
to a KS test, the component frequencies and the density; one EM step to the closed forms of a
weighted mean and variance; repeated EM to a known mixture (importance weighted, so a dropped w_n
fails); the merge to the law of total variance and to invariance under relabelling.
"""
import math

import numpy as np
import pytest

RNG = np.random.default_rng(2718)


def _model(w, mu, sigma, n=0.0):
    return dict(w=np.asarray(w, float), mu=np.asarray(mu, float), sigma=np.asarray(sigma, float), n=float(n))


def test_norm_ppf_inverts_phi(orc):
    stats = pytest.importorskip("scipy.stats")
    for p in [1e-12, 1e-6, 0.001, 0.025, 0.3, 0.5, 0.77, 0.975, 0.999999]:
        x = orc.norm_ppf(p)
        assert abs(x - stats.norm.ppf(p)) < 1e-9 * (1 + abs(x))
        assert abs(0.5 * math.erfc(-x / math.sqrt(2)) - p) < 1e-14 * max(p, 1e-3)
    assert abs(orc.norm_ppf(0.975) - 1.959963984540054) < 1e-12


def test_truncated_mixture_density(orc):
    stats = pytest.importorskip("scipy.stats")
    lo, hi = -1.0, 2.5
    m = _model([0.2, 0.5, 0.3], [-0.8, 0.4, 2.4], [0.3, 0.7, 0.2])
    x, wq = np.polynomial.legendre.leggauss(200)
    # integrate piecewise (narrow components) -> 1
    edges = np.linspace(lo, hi, 41)
    tot = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        xs = 0.5 * (b - a) * x + 0.5 * (a + b)
        tot += 0.5 * (b - a) * sum(w * math.exp(orc.gmm_lnpdf(m, lo, hi, t)) for w, t in zip(wq, xs))
    assert abs(tot - 1.0) < 1e-12
    for t in np.linspace(lo, hi, 13):
        ref = sum(m["w"][c] * stats.truncnorm.pdf(t, (lo - m["mu"][c]) / m["sigma"][c], (hi - m["mu"][c]) / m["sigma"][c],
                                                  loc=m["mu"][c], scale=m["sigma"][c]) for c in range(3))
        assert abs(orc.gmm_lnpdf(m, lo, hi, t) - math.log(ref)) < 1e-10
    # unnormalised weights mean the same model
    m2 = dict(m, w=m["w"] * 7.0)
    assert abs(orc.gmm_lnpdf(m2, lo, hi, 0.3) - orc.gmm_lnpdf(m, lo, hi, 0.3)) < 1e-14


def test_gmm_cumulative_table(orc):
    m = _model([0.25, 0.25, 0.5], [0, 0, 0], [1, 1, 1])
    cw = orc.gmm_cum(m)
    assert list(cw) == [0, 1 << 30, 1 << 31, 1 << 32]
    cw = orc.gmm_cum(_model([1.0, 2.0], [0, 0], [1, 1]))
    assert cw[0] == 0 and cw[2] == 1 << 32 and cw[1] == math.floor(2.0 ** 32 / 3)


def _sampler(orc, models, lo, hi):
    adaptive = [1 if m is not None else 0 for m in models]
    cdf = np.zeros((7, 101), np.uint64)
    for d in range(7):
        cdf[d] = orc.cdf_uniform()
    return orc.make_sampler(lo, hi, adaptive, cdf, None, 0.0, models)


def test_mixture_sampler_ks_components_and_density(orc):
    stats = pytest.importorskip("scipy.stats")
    lo = [0.0, -1.0, 0.0, -1.0, 0.0, 100.0, -0.01]
    hi = [2 * np.pi, 1.0, np.pi, 1.0, 2 * np.pi, 800.0, 0.01]
    models = [None] * 7
    models[3] = _model([0.3, 0.7], [-0.9, 0.5], [0.2, 0.3])          # cos(iota), mass piles at the edge
    models[5] = _model([0.5, 0.2, 0.3], [200.0, 450.0, 700.0], [60.0, 30.0, 150.0])  # distance
    models[6] = _model([1.0], [0.004], [0.002])                        # time, one component
    smp = _sampler(orc, models, lo, hi)
    N = 40000
    theta, lw, comp, u = orc.sample(smp, 77, 0, 0, 0, N, with_u=True)
    np.testing.assert_allclose(u[3], np.cos(theta[3]), atol=1e-12)
    np.testing.assert_allclose(u[5], theta[5], atol=0)
    lnp_ps = np.zeros(N)
    for d in (3, 5, 6):
        m = models[d]
        C = len(m["w"])
        assert np.all(comp[d] < C) and np.all((u[d] >= lo[d]) & (u[d] <= hi[d]))
        # component frequencies ~ weights (binomial, 5 sigma)
        for c in range(C):
            f = np.mean(comp[d] == c)
            assert abs(f - m["w"][c]) < 5 * math.sqrt(m["w"][c] * (1 - m["w"][c]) / N) + 1e-12
            # inside a component: its truncated normal
            a, b = (lo[d] - m["mu"][c]) / m["sigma"][c], (hi[d] - m["mu"][c]) / m["sigma"][c]
            sel = u[d][comp[d] == c]
            assert stats.kstest(sel, stats.truncnorm(a, b, loc=m["mu"][c], scale=m["sigma"][c]).cdf).pvalue > 1e-3
        lnp = np.log(3 * u[d] ** 2 / (hi[d] ** 3 - lo[d] ** 3)) if d == 5 else -np.log(hi[d] - lo[d])
        lnp_ps += lnp - np.array([orc.gmm_lnpdf(m, lo[d], hi[d], t) for t in u[d]])
    np.testing.assert_allclose(lw, lnp_ps, rtol=1e-12, atol=1e-12)
    # other dimensions: the prior, flagged 255
    assert np.all(comp[0] == 255) and np.all(comp[4] == 255)


def test_em_step_single_component_is_weighted_moments(orc):
    lo, hi = 0.0, 10.0
    u = RNG.uniform(lo, hi, 5000)
    w = RNG.exponential(size=5000)
    g = orc.gmm_em_step(_model([1.0], [3.0], [1.0]), u, w, lo, hi)
    mu = np.sum(w * u) / np.sum(w)
    var = np.sum(w * (u - mu) ** 2) / np.sum(w)
    assert abs(g["mu"][0] - mu) < 1e-12 * 10 and abs(g["sigma"][0] - math.sqrt(var)) < 1e-10
    assert g["w"][0] == 1.0
    # sigma floor: every sample at one point
    g = orc.gmm_em_step(_model([1.0], [3.0], [1.0]), np.full(10, 4.0), np.ones(10), lo, hi)
    assert g["mu"][0] == 4.0 and abs(g["sigma"][0] - 1e-3 * (hi - lo)) < 1e-15


def test_em_two_components_hand_computed(orc):
    """One EM step on three samples, worked out from the E- and M-step formulas by hand."""
    lo, hi = -5.0, 5.0
    m = _model([0.5, 0.5], [-1.0, 1.0], [1.0, 1.0])
    u = np.array([-1.0, 0.0, 2.0])
    w = np.array([1.0, 2.0, 0.5])
    g = orc.gmm_em_step(m, u, w, lo, hi)
    # responsibilities of component 0: e^{0} / (e^{0} + e^{-2}), 1/2, e^{-4.5} / (e^{-4.5} + e^{-0.5})
    r0 = np.array([1 / (1 + math.exp(-2)), 0.5, math.exp(-4.5) / (math.exp(-4.5) + math.exp(-0.5))])
    for c, r in enumerate((r0, 1 - r0)):
        q = w * r
        mu = np.sum(q * u) / np.sum(q)
        assert abs(g["mu"][c] - mu) < 1e-14
        assert abs(g["sigma"][c] - math.sqrt(np.sum(q * (u - mu) ** 2) / np.sum(q))) < 1e-13
        assert abs(g["w"][c] - np.sum(q) / np.sum(w)) < 1e-15


def test_em_recovers_target_from_importance_weights(orc):
    """Samples from a uniform proposal weighted by target / proposal: EM converges to the target
    mixture (a fit that ignored the weights would return a flat model)."""
    lo, hi = 0.0, 1.0
    true = _model([0.35, 0.65], [0.25, 0.7], [0.05, 0.08])
    N = 200000
    u = RNG.uniform(lo, hi, N)
    w = sum(true["w"][c] * np.exp(-0.5 * ((u - true["mu"][c]) / true["sigma"][c]) ** 2) / true["sigma"][c] for c in range(2))
    g = orc.gmm_init(2, lo, hi)
    for _ in range(60):
        g = orc.gmm_em_step(g, u, w, lo, hi)
    order = np.argsort(g["mu"])
    np.testing.assert_allclose(g["mu"][order], true["mu"], atol=3e-3)
    np.testing.assert_allclose(g["sigma"][order], true["sigma"], atol=3e-3)
    np.testing.assert_allclose(g["w"][order], true["w"], atol=1e-2)


def test_merge_total_variance_and_relabelling(orc):
    cur = _model([1.0], [2.0], [0.5], n=300)
    bat = _model([1.0], [3.0], [1.0])
    g = orc.gmm_merge(cur, bat, 100)
    # pooled moments of 300 points (mean 2, var .25) and 100 points (mean 3, var 1)
    mu = (300 * 2 + 100 * 3) / 400
    var = (300 * 0.25 + 100 * 1.0) / 400 + (300 * 4 + 100 * 9) / 400 - mu * mu
    assert abs(g["mu"][0] - mu) < 1e-14 and abs(g["sigma"][0] ** 2 - var) < 1e-13
    assert g["w"][0] == 1.0 and g["n"] == 400
    # relabelled batch components are matched back to the nearest current ones
    cur = _model([0.2, 0.3, 0.5], [0.0, 5.0, 10.0], [1.0, 1.0, 1.0], n=1000)
    bat = _model([0.45, 0.25, 0.3], [10.5, -0.2, 5.1], [1.2, 0.9, 1.1])
    g = orc.gmm_merge(cur, bat, 1000)
    for a, j in enumerate([2, 0, 1]):
        A, B = 1000 * cur["w"][j], 1000 * bat["w"][a]
        assert abs(g["mu"][a] - (A * cur["mu"][j] + B * bat["mu"][a]) / (A + B)) < 1e-12
        assert abs(g["w"][a] - (A + B) / 2000) < 1e-15
    # merging a model with itself keeps it and adds the counts
    g = orc.gmm_update(cur, np.zeros(5), np.ones(5), 0, -10.0, 20.0)
    np.testing.assert_allclose(g["mu"], cur["mu"], rtol=1e-15)
    np.testing.assert_allclose(g["sigma"], cur["sigma"], rtol=1e-13)
    np.testing.assert_allclose(g["w"], cur["w"], rtol=1e-15)
    assert g["n"] == 1005
    # an untrained model (n = 0) is replaced by the batch model
    fresh = orc.gmm_init(3, -10.0, 20.0)
    g = orc.gmm_merge(fresh, bat, 50)
    np.testing.assert_allclose(g["mu"], bat["mu"], rtol=1e-15)


def test_gmm_init(orc):
    g = orc.gmm_init(4, 2.0, 10.0)
    np.testing.assert_allclose(g["mu"], [3, 5, 7, 9])
    np.testing.assert_allclose(g["sigma"], [2, 2, 2, 2])
    np.testing.assert_allclose(g["w"], [0.25] * 4)
    assert g["n"] == 0.0
