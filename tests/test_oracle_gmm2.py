"""Pins of the oracle's correlated sky-pair mixture (Sec. "Adaptive sampling with gaussian mixture
models": correlated sampling in a subset of dimensions; App. "Gaussian mixture model
implementation": multivariate EM, the merge, truncation to the rectangular domain), CPU only.

Each function is tied to something other than itself: the rectangle mass to scipy's bivariate
normal CDF; the truncated pair density to 2-D quadrature over the rectangle; the sampler to the
component frequencies, a chi-square test of every component's accepted points against its cell
masses, and the density it reports; one EM step with one component to numpy's weighted mean and
covariance; repeated EM to a known correlated mixture (importance weighted, so a dropped w_n
fails); the merge to the pooled moments of two samples (law of total covariance) and to
invariance under relabelling; the floors to their definitions.
"""
import numpy as np
import pytest

LO = np.array([0.0, -1.0])
HI = np.array([2 * np.pi, 1.0])


def _pair(w, mu, cov, n=0.0):
    return dict(w=np.asarray(w, float), mu=np.asarray(mu, float).reshape(-1, 2),
                cov=np.asarray(cov, float).reshape(-1, 3), n=float(n))


def _S(c):
    return np.array([[c[0], c[1]], [c[1], c[2]]])


def test_rectangle_mass_against_scipy(orc):
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(1)
    for _ in range(12):
        mu = rng.uniform([-1.0, -1.5], [7.0, 1.5])
        s0, s1 = rng.uniform(0.05, 3.0, 2)
        rho = rng.uniform(-0.9, 0.9)
        cov = np.array([s0 * s0, rho * s0 * s1, s1 * s1])
        F = lambda x, y: stats.multivariate_normal(mu, _S(cov)).cdf([x, y])
        ref = F(HI[0], HI[1]) - F(LO[0], HI[1]) - F(HI[0], LO[1]) + F(LO[0], LO[1])
        assert abs(orc.bvn_rect(mu, cov, LO, HI) - ref) < 2e-7, (mu, cov)  # scipy's CDF is ~1e-8 accurate


def test_pair_density_integrates_to_one(orc):
    m = _pair([0.5, 0.3, 0.2], [[1.0, 0.5], [4.0, -0.7], [6.1, 0.9]],
              [[0.6, 0.2, 0.1], [1.5, -0.5, 0.3], [0.05, 0.01, 0.02]])
    Z = orc.gmm2_masses(m, LO, HI)
    x, wq = np.polynomial.legendre.leggauss(24)
    tot = 0.0
    e0, e1 = np.linspace(LO[0], HI[0], 25), np.linspace(LO[1], HI[1], 17)
    for a0, b0 in zip(e0[:-1], e0[1:]):
        xs0 = 0.5 * (b0 - a0) * x + 0.5 * (a0 + b0)
        for a1, b1 in zip(e1[:-1], e1[1:]):
            xs1 = 0.5 * (b1 - a1) * x + 0.5 * (a1 + b1)
            f = np.array([[np.exp(orc.gmm2_lnpdf(m, LO, HI, [u, v], Z)) for v in xs1] for u in xs0])
            tot += 0.25 * (b0 - a0) * (b1 - a1) * wq @ f @ wq
    assert abs(tot - 1.0) < 1e-6


def test_sampler_components_cells_and_density(orc):
    """Every component's accepted points follow its bivariate normal truncated to the rectangle:
    a chi-square test over 6 x 6 cells whose expected masses are rectangle masses of the component
    divided by its mass in the domain; the component frequencies follow the weights; ln p - ln p_s
    is the prior minus the pair density."""
    stats = pytest.importorskip("scipy.stats")
    m = _pair([0.45, 0.35, 0.2], [[1.5, 0.6], [4.5, -0.2], [0.3, -0.9]],
              [[0.8, 0.35, 0.3], [2.0, -0.8, 0.5], [0.4, 0.1, 0.1]])
    lo = [LO[0], LO[1], 0.0, -1.0, 0.0, 100.0, -1e-3]
    hi = [HI[0], HI[1], np.pi, 1.0, 2 * np.pi, 1000.0, 1e-3]
    cdf = np.stack([orc.cdf_uniform() for _ in range(7)])
    smp = orc.make_sampler(lo, hi, [1, 1, 0, 0, 0, 0, 0], cdf, pair=m)
    N = 60000
    theta, lw, bins, u = orc.sample(smp, 99, 0, 0, 0, N, with_u=True)
    comp = bins[0]
    assert np.array_equal(bins[0], bins[1])
    for c in range(3):
        k = np.count_nonzero(comp == c)
        p = m["w"][c] / m["w"].sum()
        assert abs(k - N * p) < 5 * np.sqrt(N * p * (1 - p))
        pts = u[:2, comp == c]
        assert np.all(pts[0] >= LO[0]) and np.all(pts[0] <= HI[0]) and np.all(pts[1] >= LO[1]) and np.all(pts[1] <= HI[1])
        Z = orc.bvn_rect(m["mu"][c], m["cov"][c], LO, HI)
        e0 = np.linspace(LO[0], HI[0], 7)
        e1 = np.linspace(LO[1], HI[1], 7)
        obs, exp = [], []
        for a0, b0 in zip(e0[:-1], e0[1:]):
            for a1, b1 in zip(e1[:-1], e1[1:]):
                obs.append(np.count_nonzero((pts[0] >= a0) & (pts[0] < b0) & (pts[1] >= a1) & (pts[1] < b1)))
                exp.append(pts.shape[1] * orc.bvn_rect(m["mu"][c], m["cov"][c], [a0, a1], [b0, b1]) / Z)
        obs, exp = np.array(obs), np.array(exp)
        keep = exp > 5
        chi2 = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep])
        assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4, (c, chi2, keep.sum())
    Zm = orc.gmm2_masses(m, LO, HI)
    for n in range(0, N, 997):
        want = -np.log(HI[0] - LO[0]) - np.log(HI[1] - LO[1]) - orc.gmm2_lnpdf(m, LO, HI, u[:2, n], Zm)
        assert abs(lw[n] - want) < 1e-9
    # the physical parameters: ra = u0, dec = asin(u1)
    np.testing.assert_allclose(theta[0], u[0], atol=1e-15)
    np.testing.assert_allclose(theta[1], np.arcsin(u[1]), atol=1e-12)


def test_one_component_em_step_is_weighted_mean_and_covariance(orc):
    rng = np.random.default_rng(3)
    x = np.stack([rng.uniform(1, 5, 5000), rng.uniform(-0.8, 0.9, 5000)])
    x[1] = np.clip(0.3 * (x[0] - 3) + 0.2 * rng.normal(size=5000), -1, 1)
    w = rng.exponential(size=5000)
    m = orc.gmm2_em_step(_pair([1.0], [[3.0, 0.0]], [[1.0, 0.0, 1.0]]), x[0], x[1], w, LO, HI)
    mu = np.average(x, axis=1, weights=w)
    C = np.cov(x, aweights=w, bias=True)
    np.testing.assert_allclose(m["mu"][0], mu, rtol=1e-12)
    np.testing.assert_allclose(m["cov"][0], [C[0, 0], C[0, 1], C[1, 1]], rtol=1e-10)
    assert m["w"][0] == 1.0


def test_em_recovers_a_correlated_mixture_from_weighted_uniform_points(orc):
    """Importance-weighted uniform points on the rectangle (weights = target density) fitted by
    repeated EM steps: the components' means, covariances and weights approach the target's."""
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(5)
    tw = np.array([0.6, 0.4])
    tmu = np.array([[2.0, 0.3], [4.5, -0.4]])
    tcov = np.array([[0.15, 0.05, 0.04], [0.2, -0.06, 0.05]])
    N = 200000
    x = np.stack([rng.uniform(LO[0], HI[0], N), rng.uniform(LO[1], HI[1], N)])
    dens = sum(tw[c] * stats.multivariate_normal(tmu[c], _S(tcov[c])).pdf(x.T) for c in range(2))
    m = _pair([0.5, 0.5], [[1.5, 0.0], [5.0, 0.0]], [[1.0, 0.0, 0.3], [1.0, 0.0, 0.3]])
    for _ in range(60):
        m = orc.gmm2_em_step(m, x[0], x[1], dens, LO, HI)
    np.testing.assert_allclose(m["mu"], tmu, atol=0.02)
    np.testing.assert_allclose(m["cov"], tcov, atol=0.01)
    np.testing.assert_allclose(m["w"], tw, atol=0.02)
    # without the sample weights the fit would stay near the uniform cloud
    m0 = _pair([0.5, 0.5], [[1.5, 0.0], [5.0, 0.0]], [[1.0, 0.0, 0.3], [1.0, 0.0, 0.3]])
    for _ in range(10):
        m0 = orc.gmm2_em_step(m0, x[0], x[1], np.ones(N), LO, HI)
    assert np.abs(m0["cov"][:, 0] - tcov[:, 0]).max() > 0.3


def test_floors(orc):
    rng = np.random.default_rng(7)
    t = rng.uniform(1, 5, 4000)
    x = np.stack([t, np.clip(0.5 * (t - 3), -1, 1)])  # exactly collinear: rho = 1
    m = orc.gmm2_em_step(_pair([1.0], [[3.0, 0.0]], [[1.0, 0.0, 1.0]]), x[0], x[1], np.ones(4000), LO, HI)
    c = m["cov"][0]
    assert abs(c[1]) <= 0.9 * np.sqrt(c[0] * c[2]) * (1 + 1e-12)
    x2 = np.stack([np.full(100, 2.0), np.full(100, 0.5)])  # a point mass: sigma floors
    m2 = orc.gmm2_em_step(_pair([1.0], [[3.0, 0.0]], [[1.0, 0.0, 1.0]]), x2[0], x2[1], np.ones(100), LO, HI)
    np.testing.assert_allclose(np.sqrt(m2["cov"][0][[0, 2]]), 1e-3 * (HI - LO), rtol=1e-12)


def test_merge_is_pooled_moments_and_ignores_labels(orc):
    """Two batches, each fitted by one EM step with one component per cluster; the merge of the
    second into the first (N = size of the first) equals the moments of the pooled points per
    cluster; relabelling the batch's components does not change the result."""
    rng = np.random.default_rng(9)

    def cloud(n, mu, cov):
        return rng.multivariate_normal(mu, _S(cov), n).T

    A = [cloud(3000, [1.5, 0.3], [0.1, 0.02, 0.02]), cloud(2000, [4.5, -0.3], [0.2, -0.03, 0.03])]
    B = [cloud(1500, [1.6, 0.25], [0.12, 0.01, 0.03]), cloud(2500, [4.4, -0.35], [0.15, -0.02, 0.02])]

    def fit(parts):
        x = np.concatenate(parts, axis=1)
        ws, mus, covs = [], [], []
        for p in parts:
            ws.append(p.shape[1] / x.shape[1])
            mus.append(p.mean(axis=1))
            C = np.cov(p, bias=True)
            covs.append([C[0, 0], C[0, 1], C[1, 1]])
        return _pair(ws, mus, covs, n=x.shape[1])

    cur, bat = fit(A), fit(B)
    merged = orc.gmm2_merge(cur, bat, 4000.0, LO, HI)
    for c in range(2):
        pool = np.concatenate([A[c], B[c]], axis=1)
        C = np.cov(pool, bias=True)
        np.testing.assert_allclose(merged["mu"][c], pool.mean(axis=1), rtol=1e-10)
        np.testing.assert_allclose(merged["cov"][c], [C[0, 0], C[0, 1], C[1, 1]], rtol=1e-8, atol=1e-12)
        assert abs(merged["w"][c] - pool.shape[1] / 9000.0) < 1e-12
    assert merged["n"] == 9000.0
    swapped = _pair(bat["w"][::-1], bat["mu"][::-1], bat["cov"][::-1], n=bat["n"])
    m2 = orc.gmm2_merge(cur, swapped, 4000.0, LO, HI)
    for k in ("w", "mu", "cov"):
        # component a of the output is batch component a merged with its match: same set, new order
        np.testing.assert_allclose(np.sort(m2[k].reshape(len(m2["w"]), -1), axis=0),
                                   np.sort(merged[k].reshape(len(merged["w"]), -1), axis=0), rtol=1e-12)


def test_untrained_model_takes_the_batch(orc):
    cur = orc.gmm2_init(3, LO, HI)
    bat = _pair([0.2, 0.3, 0.5], [[1.0, 0.1], [3.0, 0.2], [5.0, -0.3]],
                [[0.2, 0.01, 0.05], [0.3, 0.02, 0.04], [0.1, -0.01, 0.03]])
    out = orc.gmm2_merge(cur, bat, 1000.0, LO, HI)
    np.testing.assert_allclose(out["mu"], bat["mu"], rtol=1e-14)
    np.testing.assert_allclose(out["cov"], bat["cov"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["w"], bat["w"], rtol=1e-14)
