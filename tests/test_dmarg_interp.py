"""The distance-marginalised kernels replace per-bin table reads of ln F(a, b) by one Chebyshev
interpolant per sample and 64-bin chunk (degree 9, the 10 Chebyshev points of the chunk's data-term
range, used when the range is at most 12 wide, evaluated as a polynomial in the range's own
coordinate).  This pins the accuracy that choice relies on:
the interpolant of the exact ln F (the oracle's quadrature, App. "Distance marginalization")
stays within 1e-4 of it over such ranges, for quadratic terms b from 1e-4 to 1e4 and ranges
placed in the prior-dominated, interior and boundary regimes of the likelihood peak u = a / 2b.
CPU only; the kernels' own values are checked against the oracle by tests/test_gpu_dmarg.py."""
import numpy as np
import pytest

D_MIN, D_MAX, D_REF = 100.0, 1000.0, 100.0
NODES, WMAX = 10, 12.0


def _interp(f, lo, hi, dtype=np.float64):
    """The kernels' construction: nodes mid + half cos(pi (k + 1/2) / 10), Chebyshev coefficients
    c_j = (2 - [j = 0]) / 10 sum_k f_k T_j(x_k), monomial coefficients m_i = sum_j a_ij c_j of t =
    (a - mid) / half, Horner evaluation -- in FP64, or step by step in FP32 as the kernels do."""
    F = dtype
    mid, half = F(0.5) * (F(lo) + F(hi)), max(F(0.5) * (F(hi) - F(lo)), F(0.5))
    k = np.arange(NODES)
    x = np.cos(np.pi * (k + 0.5) / NODES).astype(F)
    fk = np.array([f(float(F(half) * xi + mid)) for xi in x]).astype(F)
    T = np.array([[(1.0 if j == 0 else 2.0) / NODES * np.cos(j * np.pi * (kk + 0.5) / NODES) for kk in k]
                  for j in range(NODES)]).astype(F)
    c = np.array([F(np.sum(T[j] * fk, dtype=F)) for j in range(NODES)], dtype=F)
    a_ij = np.zeros((NODES, NODES))
    for j in range(NODES):
        p = np.polynomial.chebyshev.cheb2poly([0] * j + [1])
        a_ij[:len(p), j] = p
    m = np.array([F(np.sum(a_ij[i].astype(F) * c, dtype=F)) for i in range(NODES)], dtype=F)
    inv_half = F(1) / half

    def ev(a):
        t = (F(a) - mid) * inv_half
        v = m[-1]
        for i in range(NODES - 2, -1, -1):
            v = F(v * t + m[i])
        return float(v)
    return ev


def test_interpolant_reproduces_polynomials():
    """Interpolation at 10 points is exact for polynomials of degree <= 9 (a check of the
    coefficient formula and the recurrence)."""
    rng = np.random.default_rng(0)
    p = np.polynomial.Polynomial(rng.normal(size=NODES))
    ev = _interp(p, -3.0, 5.0)
    a = np.linspace(-3.0, 5.0, 41)
    assert np.abs(np.array([ev(x) for x in a]) - p(a)).max() < 1e-9 * np.abs(p(a)).max()


@pytest.mark.parametrize("b", [1e-4, 0.05, 0.5, 1.0, 2.0, 3.0, 6.0, 12.0, 100.0, 1e4])
def test_interpolant_of_lnF_within_1e_4(orc, b):
    f = lambda a: orc.dmarg_lnF(a, b, D_MIN, D_MAX, D_REF)
    rng = np.random.default_rng(int(b * 1000) % 2**32)
    worst = 0.0
    for c0 in (0.0, 0.2 * b, b, 2.0 * b, rng.uniform(-3, 3) * max(1.0, np.sqrt(2 * b)) + 1.0 * b):
        lo, hi = c0 - WMAX / 2, c0 + WMAX / 2
        ev = _interp(f, lo, hi)
        for a in np.linspace(lo, hi, 25):
            worst = max(worst, abs(ev(a) - f(a)))
    assert worst < 1e-4, worst


@pytest.mark.parametrize("b", [0.05, 1.0, 3.0, 12.0, 100.0])
def test_fp32_construction_within_6e_5(orc, b):
    """The same construction in FP32 arithmetic (nodes, coefficients, Horner) for data terms below
    2000 in size, against ln F at the FP32 data term."""
    f = lambda a: orc.dmarg_lnF(a, b, D_MIN, D_MAX, D_REF)
    worst = 0.0
    for c0 in (0.0, 0.2 * b, b, 2.0 * b):
        for W in (1.0, 6.0, WMAX):
            lo, hi = c0 - W / 2, c0 + W / 2
            ev = _interp(f, lo, hi, np.float32)
            for a in np.linspace(lo, hi, 17):
                a32 = float(np.float32(a))
                worst = max(worst, abs(ev(a32) - f(a32)))
    assert worst < 6e-5, worst
