"""Pins of the oracle's distance marginalisation (CPU only).

ln F(a, b) = ln int p(D) exp(a x - b x^2) dD (x = D_ref / D, p prop. to D^2 on [D_min, D_max]) is
tied to an independent adaptive quadrature in D, and the distance-marginalised likelihood to a
direct quadrature over D of the (pinned) time-marginalised likelihood exp(lnL_t(theta, D)).
"""
import math

import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

D_MIN, D_MAX, D_REF = 100.0, 1000.0, 100.0


def test_lnF_normalisation_and_adaptive_quadrature(orc):
    integrate = pytest.importorskip("scipy.integrate")
    assert abs(orc.dmarg_lnF(0.0, 0.0, D_MIN, D_MAX, D_REF)) < 1e-13  # normalised prior
    norm = 3.0 / (D_MAX ** 3 - D_MIN ** 3)
    for a, b in [(5.0, 3.0), (-20.0, 2.0), (300.0, 150.0), (60.0, 0.5), (2000.0, 1500.0), (1.0, 1e-4), (0.0, 40.0),
                 (1e4, 1e4), (2.2e4, 1e4), (100.0, 600.0)]:
        x0 = min(max(a / (2 * b), D_REF / D_MAX), D_REF / D_MIN)
        shift = a * x0 - b * x0 * x0
        f = lambda D: norm * D * D * math.exp(a * D_REF / D - b * (D_REF / D) ** 2 - shift)
        peak = D_REF / x0
        val, err = integrate.quad(f, D_MIN, D_MAX, points=[peak], limit=400, epsabs=0, epsrel=1e-12)
        ref = shift + math.log(val)
        assert abs(orc.dmarg_lnF(a, b, D_MIN, D_MAX, D_REF) - ref) < 1e-9, (a, b)


@pytest.mark.parametrize("shape", ["hl_m2", "hlv_m9"])
def test_dmarg_equals_distance_integral_of_lnL_t(orc, shape):
    """exp(lnL_dmarg(theta)) = int p(D) exp(lnL_t(theta, D)) dD, the right side from the pinned
    time-marginalised likelihood on a 400-node Gauss-Legendre rule in D."""
    if shape == "hl_m2":
        point = S.workload_point(S.SMALL)
    else:
        point = S.make_point(S.SEED_BASE + 70, 3, 9, 64, spectrum="decay")
    th = S.workload_samples(S.SMALL, 6)
    got = orc.lnL_dmarg(point, th, D_MIN, D_MAX)
    xg, wg = np.polynomial.legendre.leggauss(400)
    D = 0.5 * (D_MAX - D_MIN) * xg + 0.5 * (D_MAX + D_MIN)
    w = 0.5 * (D_MAX - D_MIN) * wg * 3.0 * D ** 2 / (D_MAX ** 3 - D_MIN ** 3)
    for n in range(th.shape[1]):
        t = np.repeat(th[:, n:n + 1], D.size, axis=1)
        t[5] = D
        lt = orc.lnL_t(point, t)
        m = lt.max()
        ref = m + math.log(np.sum(w * np.exp(lt - m)))
        assert abs(got[n] - ref) < 1e-8, (n, got[n], ref)


def test_dmarg_ignores_sample_distance(orc):
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 8)
    t2 = th.copy()
    t2[5] = np.linspace(150, 900, 8)
    np.testing.assert_array_equal(orc.lnL_dmarg(point, th, D_MIN, D_MAX), orc.lnL_dmarg(point, t2, D_MIN, D_MAX))
