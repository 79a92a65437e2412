"""Pins of the oracle's analytic gradient of lnL_t (the adjoint the GPU gradient is checked
against), on the CPU.

The gradient is tied to the oracle's forward lnL_t, which is itself pinned by the likelihood
tests: central finite differences in every extrinsic parameter, directional differences in Q,
U and V, the closed form of the distance derivative (the data term scales as 1/D, <h|h>/2 as
1/D^2) and the derivative of a closed-form Wigner-d element.
"""
import math

import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

H = np.array([1e-6, 1e-6, 1e-6, 1e-6, 1e-6, 1e-6, 1e-8])  # relative for D, seconds for t_c


def test_wigner_d_deriv_closed_form_and_differences(orc):
    for beta in (0.3, 1.1, 2.7):
        # d^2_{2,2} = cos^4(beta/2), d^2_{1,2} = +2 cos^3(beta/2) sin(beta/2)
        c, s = math.cos(beta / 2), math.sin(beta / 2)
        assert abs(orc.wigner_d_deriv(2, 2, 2, beta) + 2 * c ** 3 * s) < 1e-14
        ref12 = 2 * (-1.5 * c * c * s * s + 0.5 * c ** 4)
        assert abs(orc.wigner_d_deriv(2, 1, 2, beta) - ref12) < 1e-14
        h = 1e-6
        for l in (2, 3, 4):
            for m in range(-l, l + 1):
                fd = (orc.wigner_d(l, m, 2, beta + h) - orc.wigner_d(l, m, 2, beta - h)) / (2 * h)
                assert abs(orc.wigner_d_deriv(l, m, 2, beta) - fd) < 1e-8


def _bins(point, th, orc):
    """floor of the fractional interpolation position per detector (the same for every j)."""
    x = []
    for k in range(point.det_pos.shape[0]):
        dt = orc.delay(point.det_pos[k], th[0], th[1], point.gmst)
        x.append(math.floor((th[6] - 0.5 * point.n_window / point.fs + dt - point.t_start) * point.fs))
    return x


@pytest.mark.parametrize("wl,M", [(S.SMALL, None), (S.FULL, 9)])
def test_grad_theta_matches_central_differences(orc, wl, M):
    c = S.WORKLOADS[wl]
    point = S.make_point(S.SEED_BASE + 40 + c["seed"], c["n_det"], M or c["n_modes"], 64, spectrum=c["spectrum"])
    th = S.prior_samples(np.random.default_rng(41 + c["seed"]), 24)
    lnl, g, _, _, _ = orc.lnL_t_grad(point, th)
    np.testing.assert_allclose(lnl, orc.lnL_t(point, th), rtol=1e-13, atol=1e-12)
    checked = 0
    for n in range(th.shape[1]):
        for d in range(7):
            h = H[d] * (th[5, n] if d == 5 else 1.0)
            tp, tm = th[:, n].copy(), th[:, n].copy()
            tp[d] += h
            tm[d] -= h
            if _bins(point, tp, orc) != _bins(point, tm, orc):
                continue  # a kink of the linear interpolation lies inside the step
            fd = (orc.lnL_t(point, tp[:, None])[0] - orc.lnL_t(point, tm[:, None])[0]) / (2 * h)
            scale = max(1.0, abs(fd), abs(lnl[n]) * (1.0 / th[5, n] if d == 5 else 1.0))
            assert abs(g[d, n] - fd) < 2e-6 * scale, (n, d, g[d, n], fd)
            checked += 1
    assert checked >= 7 * th.shape[1] - 6


def test_grad_distance_closed_form(orc):
    """d lnL_t/dD = (2A - sum_j pi_j data_j)/D with pi the softmax of lnL(j)."""
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 16)
    _, g, _, _, _ = orc.lnL_t_grad(point, th)
    for n in range(th.shape[1]):
        lnL, data, A = orc.lnL_grid(point, th[:, n])
        p = np.exp(lnL - lnL.max())
        p /= p.sum()
        ref = (2 * A - p @ data) / th[5, n]
        assert abs(g[5, n] - ref) < 1e-12 * max(1.0, abs(ref))


def _perturbed(point, **kw):
    import dataclasses
    return dataclasses.replace(point, **kw)


def test_grad_QUV_directional_differences(orc):
    point = S.make_point(S.SEED_BASE + 50, 3, 5, 64, spectrum="decay")
    th = S.prior_samples(np.random.default_rng(51), 8)
    wts = np.random.default_rng(52).normal(size=th.shape[1])
    _, _, gQ, gU, gV = orc.lnL_t_grad(point, th, wts)
    rng = np.random.default_rng(53)

    def f(pt):
        return wts @ orc.lnL_t(pt, th)

    for name, grad in (("Q", gQ), ("U", gU), ("V", gV)):
        base = getattr(point, name)
        dirn = rng.normal(size=base.shape) + 1j * rng.normal(size=base.shape)
        h = 1e-5
        fd = (f(_perturbed(point, **{name: base + h * dirn})) - f(_perturbed(point, **{name: base - h * dirn}))) / (2 * h)
        an = np.sum(grad[..., 0] * dirn.real + grad[..., 1] * dirn.imag)
        assert abs(an - fd) < 1e-6 * max(1.0, abs(fd)), (name, an, fd)


def test_grad_upstream_weights_are_linear(orc):
    """g_theta scales per sample with the upstream weight; g_Q, g_U, g_V are weighted sums."""
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 6)
    w = np.array([0.5, -2.0, 0.0, 1.0, 3.0, -0.25])
    _, g1, _, _, _ = orc.lnL_t_grad(point, th)
    _, gw, qw, uw, vw = orc.lnL_t_grad(point, th, w)
    np.testing.assert_allclose(gw, g1 * w[None, :], rtol=1e-14, atol=0)
    q = np.zeros_like(qw)
    u = np.zeros_like(uw)
    v = np.zeros_like(vw)
    for n in range(th.shape[1]):
        _, _, qn, un, vn = orc.lnL_t_grad(point, th[:, n:n + 1])
        q += w[n] * qn
        u += w[n] * un
        v += w[n] * vn
    np.testing.assert_allclose(qw, q, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(uw, u, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(vw, v, rtol=1e-12, atol=1e-14)
