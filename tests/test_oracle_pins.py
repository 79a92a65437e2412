"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties one oracle function to something other than itself: a closed form, an
invariant, a textbook average, an independent library, or a direct evaluation of the likelihood
from its definition -<h-d|h-d>/2 in the frequency domain (Eq. (eq:loglikelihood) with
Eq. (eq:QUV)).  A dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.
"""
import math

import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

RNG = np.random.default_rng(12345)


# ------------------------------------------------------------------------------ S1 geometry
def test_frame_orthonormal_and_handedness(orc):
    for _ in range(50):
        ra, dec, psi, g = RNG.uniform(0, 2 * np.pi), np.arcsin(RNG.uniform(-1, 1)), RNG.uniform(0, np.pi), RNG.uniform(0, 6)
        X, Y, n = orc.frame(ra, dec, psi, g)
        for v in (X, Y, n):
            assert abs(np.dot(v, v) - 1) < 1e-14
        assert abs(X @ Y) < 1e-14 and abs(X @ n) < 1e-14 and abs(Y @ n) < 1e-14
        np.testing.assert_allclose(np.cross(X, Y), -n, atol=1e-14)


def test_antenna_sky_average_one_fifth(orc):
    """Sky- and polarisation-averaged F+^2 = Fx^2 = 1/5 for a 90-degree interferometer."""
    D = S.detector_arrays(1)[0][0]
    xd, wd = np.polynomial.legendre.leggauss(48)
    dec = 0.5 * np.pi * xd
    wdec = 0.5 * np.pi * wd * np.cos(dec) / 2.0  # integrates cos(dec)/2 over [-pi/2, pi/2] -> 1
    ras = np.arange(12) * 2 * np.pi / 12
    psis = np.arange(8) * np.pi / 8
    fp2 = fx2 = 0.0
    for d, w in zip(dec, wdec):
        for ra in ras:
            for psi in psis:
                F = orc.antenna(D, ra, d, psi)
                fp2 += w * F.real ** 2
                fx2 += w * F.imag ** 2
    norm = len(ras) * len(psis)
    assert abs(fp2 / norm - 0.2) < 1e-12
    assert abs(fx2 / norm - 0.2) < 1e-12


def test_antenna_overhead_unit_response(orc):
    """A source at the zenith of the arm plane has |F| = 1 for every polarisation angle."""
    tens, _ = S.detector_arrays(4)
    for name, D in zip(S.NETWORK, tens):
        _, u, v = (np.array(x) for x in S.DETECTORS[name])
        z = np.cross(u, v)
        z /= np.linalg.norm(z)
        dec = math.asin(z[2])
        g = math.atan2(-z[1], z[0])  # n = (cos d cos g, -cos d sin g, sin d), g = gmst - ra
        for gmst in (0.0, 1.3):
            ra = gmst - g
            for psi in np.linspace(0, np.pi, 7):
                assert abs(abs(orc.antenna(D, ra, dec, psi, gmst)) - 1.0) < 1e-9


def test_antenna_polarisation_symmetry_and_gmst(orc):
    D = S.detector_arrays(3)[0][2]
    for _ in range(30):
        ra, dec, psi = RNG.uniform(0, 2 * np.pi), np.arcsin(RNG.uniform(-1, 1)), RNG.uniform(0, np.pi)
        F = orc.antenna(D, ra, dec, psi)
        assert abs(orc.antenna(D, ra, dec, psi + np.pi) - F) < 1e-13
        assert abs(orc.antenna(D, ra, dec, psi + np.pi / 2) + F) < 1e-13
        assert abs(orc.antenna(D, ra + 0.4, dec, psi, 0.4) - F) < 1e-13


def test_delay_triangulation(orc):
    _, pos = S.detector_arrays(2)
    base = pos[0] - pos[1]
    assert abs(np.linalg.norm(base) / S.C_SI - 10.0e-3) < 0.05e-3  # H-L light travel time
    bound = np.linalg.norm(base) / S.C_SI
    for _ in range(200):
        ra, dec = RNG.uniform(0, 2 * np.pi), np.arcsin(RNG.uniform(-1, 1))
        d = orc.delay(pos[0], ra, dec) - orc.delay(pos[1], ra, dec)
        assert abs(d) <= bound * (1 + 1e-12)
    # a source along the baseline (from L towards H) reaches H first by exactly |r_H - r_L|/c
    b = base / np.linalg.norm(base)
    dec, g = math.asin(b[2]), math.atan2(-b[1], b[0])
    d = orc.delay(pos[0], -g, dec) - orc.delay(pos[1], -g, dec)
    assert abs(d + bound) < 1e-15
    assert orc.delay(np.zeros(3), 1.0, 0.3) == 0.0


# ------------------------------------------------------------------------------ S2 harmonics
def test_sylm_l2_closed_forms(orc):
    c5 = math.sqrt(5 / (64 * math.pi))
    for iota in np.linspace(0, np.pi, 9):
        for phi in (0.0, 0.7, 2.9):
            ci, si = math.cos(iota), math.sin(iota)
            want = {
                (2, 2): c5 * (1 + ci) ** 2 * np.exp(2j * phi),
                (2, -2): c5 * (1 - ci) ** 2 * np.exp(-2j * phi),
                (2, 1): math.sqrt(5 / (16 * math.pi)) * si * (1 + ci) * np.exp(1j * phi),
                (2, -1): math.sqrt(5 / (16 * math.pi)) * si * (1 - ci) * np.exp(-1j * phi),
                (2, 0): math.sqrt(15 / (32 * math.pi)) * si ** 2,
            }
            for (l, m), w in want.items():
                assert abs(orc.sylm(l, m, iota, phi) - w) < 1e-15


def test_sylm_orthonormal_all_21_modes(orc):
    x, w = np.polynomial.legendre.leggauss(40)
    iotas = np.arccos(x)
    phis = np.arange(32) * 2 * np.pi / 32
    modes = S.ALL_MODES
    Y = np.array([[[orc.sylm(l, m, io, ph) for ph in phis] for io in iotas] for (l, m) in modes])
    G = np.einsum("aip,bip,i->ab", Y, Y.conj(), w) * (2 * np.pi / len(phis))
    np.testing.assert_allclose(G, np.eye(len(modes)), atol=1e-13)


def test_wigner_d_matches_sympy(orc):
    sp = pytest.importorskip("sympy")
    from sympy.physics.quantum.spin import Rotation
    for beta in (0.3, 1.9):
        for l in (2, 3, 4):
            for m1 in range(-l, l + 1):
                for m2 in (-2, 2, 1):
                    ref = complex(sp.N(Rotation.d(l, m1, m2, beta).doit(), 20))
                    assert abs(orc.wigner_d(l, m1, m2, beta) - ref.real) < 1e-14


# ------------------------------------------------------------------------------ S3-S5 likelihood
def orc_module():
    import oracle
    return oracle


def _fd_setup(seed, K=2, M=3, L=512, fs=4096.0, Nt=32, T_ext=128):
    """Synthetic modes h_lm, PSDs and data; Q, U, V straight from Eq. (eq:QUV)."""
    rng = np.random.default_rng(seed)
    dt, df = 1.0 / fs, fs / L
    f = np.fft.fftfreq(L, dt)
    env = np.exp(-0.5 * (f / 300.0) ** 2)
    lm = S.ALL_MODES[:M]
    hf = (rng.normal(size=(M, L)) + 1j * rng.normal(size=(M, L))) * env  # h~_lm(f), two-sided
    psd = 1.0 + rng.uniform(0.5, 2.0) * (f / 500.0) ** 2 + 0.1 * rng.uniform(size=(K, 1))
    d_t = rng.normal(size=(K, L)) * 3.0  # arbitrary real data per detector
    d_f = np.fft.fft(d_t, axis=1) * dt

    t_start = -(T_ext // 2) / fs
    # Q, U, V from the oracle's Eq. (eq:QUV); the decomposition test below then ties them (and the
    # likelihood built on them) to inner products of the full waveform with the data
    Q, U, V = orc_module().quv_from_modes(hf, psd, d_f, df, -1.0, t_start, fs, T_ext)  # every bin
    tens, _ = S.detector_arrays(K)
    point = S.Point(lm=np.array(lm, np.int32), det_tensor=tens, det_pos=np.zeros((K, 3)), Q=Q, U=U, V=V,
                    t_start=t_start, fs=fs, n_window=Nt)
    return point, dict(hf=hf, psd=psd, d_f=d_f, f=f, dt=dt, df=df, lm=lm)


def _direct_lnL(orc, aux, theta, t_arrival):
    """sum_k <h_k|d_k> - <h_k|h_k>/2 with h_k(t) = (D_ref/D) Re[F_k sum_lm Y_lm h_lm(t - t_k)]."""
    ra, dec, psi, iota, phi, dist, _ = theta
    hf, psd, d_f, f, df = aux["hf"], aux["psd"], aux["d_f"], aux["f"], aux["df"]
    tens, _ = S.detector_arrays(psd.shape[0])
    total = 0.0
    for k in range(psd.shape[0]):
        F = orc.antenna(tens[k], ra, dec, psi)
        Ylm = np.array([orc.sylm(l, m, iota, phi) for (l, m) in aux["lm"]])
        shifted = hf * np.exp(-2j * np.pi * f * t_arrival)[None, :]
        comb_f = (F * Ylm) @ shifted  # FT of F sum Y h_lm(t - t_k)
        # FT of Re[x(t)] = (x~(f) + conj(x~(-f))) / 2
        hk_f = (S.D_REF / dist) * 0.5 * (comb_f + np.conj(comb_f[(-np.arange(len(f))) % len(f)]))
        total += (2.0 * np.sum(hk_f.conj() * d_f[k] / psd[k]) * df).real
        total -= 0.5 * (2.0 * np.sum(np.abs(hk_f) ** 2 / psd[k]) * df).real
    return total


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_decomposition_equals_direct_inner_products(orc, seed):
    """Eq. (eq:loglikelihood): the Q/U/V decomposition equals <h|d> - <h|h>/2 evaluated directly."""
    point, aux = _fd_setup(seed)
    rng = np.random.default_rng(100 + seed)
    for _ in range(4):
        theta = np.array([rng.uniform(0, 2 * np.pi), np.arcsin(rng.uniform(-1, 1)), rng.uniform(0, np.pi),
                          np.arccos(rng.uniform(-1, 1)), rng.uniform(0, 2 * np.pi), rng.uniform(100, 1000),
                          rng.integers(-4, 5) / point.fs])
        lnL, data, A = orc.lnL_grid(point, theta)
        for j in (0, 7, point.n_window // 2, point.n_window - 1):
            t_arr = theta[6] + (j - point.n_window / 2) / point.fs
            ref = _direct_lnL(orc, aux, theta, t_arr)
            assert abs(lnL[j] - ref) < 1e-9 * max(1.0, abs(ref)), (j, lnL[j], ref)


def _flat_injection(orc, seed, K=3, M=5, Nt=64):
    """Noise-free, flat-profile data whose true signal is theta0 (c0 and arrival times from the oracle)."""
    rng = np.random.default_rng(seed)
    tens, pos = S.detector_arrays(K)
    theta0 = np.array([1.1, 0.4, 0.7, 0.9, 2.1, 300.0, 0.0])
    lm = S.mode_list(M)
    c0 = np.array([[(S.D_REF / theta0[5]) * orc.antenna(tens[k], *theta0[:3]) * orc.sylm(l, m, theta0[3], theta0[4])
                    for (l, m) in lm] for k in range(K)])
    point = S.make_point(int(rng.integers(1 << 30)), K, M, Nt, c_true=c0, t_true=np.zeros(K), noise=0.0,
                         pulse_sigma=None)
    return point, theta0


def test_injection_identity_and_cauchy_schwarz(orc):
    point, theta0 = _flat_injection(orc, 7)
    lnL0, data0, A0 = orc.lnL_grid(point, theta0)
    np.testing.assert_allclose(lnL0, A0, rtol=1e-12)  # lnL(theta0) = <h0|h0>/2 = A(theta0)
    np.testing.assert_allclose(data0, 2 * A0, rtol=1e-12)
    rng = np.random.default_rng(8)
    th = S.prior_samples(rng, 200)
    for n in range(th.shape[1]):
        lnL, _, _ = orc.lnL_grid(point, th[:, n])
        assert np.all(lnL <= A0 * (1 + 1e-12))
    # at fixed angles lnL(D) = a/D - b/D^2 peaks at the true distance
    for fac in (0.98, 1.02, 0.999, 1.001):
        t = theta0.copy()
        t[5] *= fac
        assert orc.lnL_grid(point, t)[0][0] < lnL0[0]


def test_symmetries_and_distance_scaling(orc):
    point = S.workload_point(S.SMALL)
    rng = np.random.default_rng(9)
    th = S.prior_samples(rng, 20)
    for n in range(th.shape[1]):
        t = th[:, n].copy()
        lnL, data, A = orc.lnL_grid(point, t)
        t2 = t.copy(); t2[2] += np.pi / 2
        _, data2, A2 = orc.lnL_grid(point, t2)
        np.testing.assert_allclose(data2, -data, rtol=1e-10, atol=1e-12)
        assert abs(A2 - A) < 1e-12 * max(1, A)
        t3 = t.copy(); t3[2] += np.pi
        _, data3, A3 = orc.lnL_grid(point, t3)
        np.testing.assert_allclose(data3, data, rtol=1e-10, atol=1e-12)
        t4 = t.copy(); t4[5] *= 2.0
        _, data4, A4 = orc.lnL_grid(point, t4)
        np.testing.assert_allclose(data4, 0.5 * data, rtol=1e-12, atol=1e-14)
        assert abs(A4 - 0.25 * A) < 1e-12 * max(1, A)
        assert A > 0


def test_time_marginalisation_logsumexp(orc):
    scipy_special = pytest.importorskip("scipy.special")
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 64)
    out = orc.lnL_t(point, th)
    for n in range(th.shape[1]):
        lnL, _, _ = orc.lnL_grid(point, th[:, n])
        ref = scipy_special.logsumexp(lnL) - math.log(point.n_window)
        assert abs(out[n] - ref) < 1e-12
    # flat profile: lnL_t equals the (j-independent) lnL
    flat, theta0 = _flat_injection(orc, 11)
    lnL, _, _ = orc.lnL_grid(flat, theta0)
    assert abs(orc.lnL_t(flat, theta0[:, None])[0] - lnL[0]) < 1e-12


def test_range_error(orc):
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 4)
    th[6, 1] = 0.05  # t_c far outside the window
    with pytest.raises(orc.RangeError):
        orc.lnL_t(point, th)


# ------------------------------------------------------------------------------ S6 Monte Carlo
def test_mc_stats_constant_and_definitions(orc):
    st = orc.mc_stats(np.full(1000, -3.5))
    assert abs(st["ln_I"] + 3.5) < 1e-14 and st["sigma_ln"] == 0.0
    assert abs(st["n_eff"] - 1000) < 1e-9 and abs(st["ess"] - 1000) < 1e-9
    lnw = RNG.normal(0, 1.5, 5000)
    w = np.exp(lnw)
    st = orc.mc_stats(lnw)
    assert abs(st["ln_I"] - math.log(w.mean())) < 1e-12
    assert abs(st["n_eff"] - w.sum() / w.max()) < 1e-9 * st["n_eff"]          # Eq. (eq:neff)
    assert abs(st["ess"] - w.sum() ** 2 / (w ** 2).sum()) < 1e-9 * st["ess"]  # Eq. (eq:neff_ESS)
    assert abs(st["sigma_ln"] - w.std(ddof=1) / math.sqrt(w.size) / w.mean()) < 1e-12
    # log space survives amplitudes far past the raw-double limit (rho ~ 37.5 in the paper)
    st = orc.mc_stats(lnw + 0.5 * 60.0 ** 2 * 2)
    assert np.isfinite(st["ln_I"]) and abs(st["ln_I"] - 3600 - math.log(w.mean())) < 1e-9


def test_toy_reweighting_model(orc):
    """Appendix toy: L = 1, p = 1, p_s = alpha x^(alpha-1); mean weight -> 1, median n_eff formula."""
    alpha, N = 3.0, 20000
    rng = np.random.default_rng(21)
    neffs, lnIs, sig = [], [], []
    for _ in range(41):
        x = rng.uniform(size=N) ** (1 / alpha)
        lnw = -math.log(alpha) - (alpha - 1) * np.log(x)
        st = orc.mc_stats(lnw)
        neffs.append(st["n_eff"]); lnIs.append(st["ln_I"]); sig.append(st["sigma_ln"])
    assert abs(np.mean(lnIs)) < 4 * np.mean(sig) / math.sqrt(len(lnIs)) + 0.01
    pred = N * alpha * (N / math.log(2)) ** (-(alpha - 1) / alpha)
    assert 0.7 < np.median(neffs) / pred < 1.4


def test_distance_only_integral_matches_quadrature(orc):
    integrate = pytest.importorskip("scipy.integrate")
    point, theta0 = _flat_injection(orc, 13, K=2, M=2, Nt=16)
    # flat profile -> lnL_t(D) = a x - b x^2 with x = D_ref / D
    _, data, A = orc.lnL_grid(point, np.r_[theta0[:5], S.D_REF, 0.0])
    a, b = data[0], A
    norm = (S.D_MAX ** 3 - S.D_MIN ** 3) / 3.0
    val, _ = integrate.quad(lambda D: math.exp(a * S.D_REF / D - b * (S.D_REF / D) ** 2) * D * D / norm,
                            S.D_MIN, S.D_MAX, epsabs=0, epsrel=1e-12)
    rng = np.random.default_rng(5)
    N = 20000
    th = np.repeat(np.r_[theta0[:5], 0.0, 0.0][:, None], N, axis=1)
    th[5] = np.cbrt(S.D_MIN ** 3 + rng.uniform(size=N) * (S.D_MAX ** 3 - S.D_MIN ** 3))
    st = orc.mc_stats(orc.lnL_t(point, th))
    assert abs(st["ln_I"] - math.log(val)) < 4 * st["sigma_ln"] + 1e-12


# ------------------------------------------------------------------------------ S0 sampler
def test_philox_statistics(orc):
    words = np.concatenate([orc.philox([n, 7, 3, 0], [0x1234, 0x5678]) for n in range(8192)])
    counts = np.bincount(words >> 24, minlength=256)
    chi2 = ((counts - words.size / 256) ** 2 / (words.size / 256)).sum()
    assert chi2 < 256 + 6 * math.sqrt(2 * 256)
    # one flipped counter bit changes about half of the 128 output bits
    ham = []
    for n in range(256):
        a = orc.philox([n, 0, 0, 0], [1, 2])
        b = orc.philox([n ^ (1 << (n % 32)), 0, 0, 0], [1, 2])
        ham.append(sum(bin(int(x ^ y)).count("1") for x, y in zip(a, b)))
    assert abs(np.mean(ham) - 64) < 2.0
    assert not np.array_equal(orc.philox([1, 0, 0, 0], [0, 0]), orc.philox([1, 0, 0, 0], [1, 0]))


def philox_kat_vectors():
    """The published Philox4x32-10 known-answer vectors in tests/golden (counter, key, expected)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    out = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        assert f[0] == "philox4x32" and f[1] == "10"
        w = [int(x, 16) for x in f[2:]]
        out.append((w[0:4], w[4:6], w[6:10]))
    return out


def test_philox_known_answer_vectors(orc):
    """The oracle's generator reproduces the Random123 known-answer vectors of Philox4x32-10 (a
    wrong multiplier, Weyl constant, round count or word order fails these, not the statistics)."""
    kat = philox_kat_vectors()
    assert len(kat) == 3
    for ctr, key, want in kat:
        assert [int(x) for x in orc.philox(ctr, key)] == want, (ctr, key)


def _sampler(orc, rng, adaptive):
    lo = [0.0, -1.0, 0.0, -1.0, 0.0, S.D_MIN, -4 / S.FS]
    hi = [2 * np.pi, 1.0, np.pi, 1.0, 2 * np.pi, S.D_MAX, 4 / S.FS]
    cdf = np.zeros((7, 101), np.uint64)
    for d in range(7):
        h = rng.gamma(0.5, size=100)
        cdf[d] = orc.cdf_from_hist(h, 0.1)
    return orc.make_sampler(lo, hi, adaptive, cdf), lo, hi, cdf


def test_sampler_histogram_ks_and_density(orc):
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(31)
    adaptive = [1, 1, 0, 1, 0, 1, 0]
    smp, lo, hi, cdf = _sampler(orc, rng, adaptive)
    N = 40000
    theta, lw, bins = orc.sample(smp, 99, 0, 0, 0, N)
    u = theta.copy(); u[1] = np.sin(theta[1]); u[3] = np.cos(theta[3])
    mass = np.diff(cdf.astype(np.float64), axis=1) / 2.0 ** 32
    lnp_ps = np.zeros(N)
    for d in range(7):
        edges = np.linspace(lo[d], hi[d], 101)
        if adaptive[d]:
            cdf_f = np.concatenate([[0.0], np.cumsum(mass[d])])
            F = lambda x, d=d, cdf_f=cdf_f, edges=edges: np.interp(x, edges, cdf_f)
            assert np.all(bins[d] == np.clip(np.searchsorted(edges, u[d], side="right") - 1, 0, 99))
            width = (hi[d] - lo[d]) / 100
            lnp = -np.log(hi[d] - lo[d]) if d != 5 else np.log(3 * u[d] ** 2 / (hi[d] ** 3 - lo[d] ** 3))
            lnp_ps += lnp - (np.log(mass[d][bins[d]]) - math.log(width))
        elif d == 5:
            F = lambda x, d=d: (x ** 3 - lo[d] ** 3) / (hi[d] ** 3 - lo[d] ** 3)
        else:
            F = lambda x, d=d: (x - lo[d]) / (hi[d] - lo[d])
        assert stats.kstest(u[d], F).pvalue > 1e-3, d
        assert np.all((u[d] >= lo[d]) & (u[d] <= hi[d]))
    np.testing.assert_allclose(lw, lnp_ps, rtol=1e-9, atol=1e-9)
    # the same counters give the same samples; another iteration gives different ones
    t2, _, _ = orc.sample(smp, 99, 0, 0, 100, 50)
    np.testing.assert_array_equal(t2, theta[:, 100:150])
    t3, _, _ = orc.sample(smp, 99, 1, 0, 100, 50)
    assert not np.allclose(t3, theta[:, 100:150])


def test_histogram_and_cdf_tables(orc):
    lnw = np.full(10, -2.0)
    b = np.array([3] * 10, np.uint8)
    h = orc.hist(lnw, b)
    assert h[3] == 1.0 and h.sum() == 1.0
    lnw = RNG.normal(size=1000)
    b = RNG.integers(0, 100, 1000).astype(np.uint8)
    h = orc.hist(lnw, b)
    ref = np.bincount(b, weights=np.exp(lnw), minlength=100)
    np.testing.assert_allclose(h, ref / ref.sum(), rtol=1e-12)
    u = orc.cdf_uniform()
    assert u[0] == 0 and u[100] == 1 << 32 and np.all(np.diff(u.astype(np.int64)) >= 42949672)
    c = orc.cdf_from_hist(np.ones(100), 0.1)
    assert np.all(np.abs(c.astype(np.int64) - u.astype(np.int64)) <= 1)
    c = orc.cdf_from_hist(np.r_[1.0, np.zeros(99)], 0.1)
    m = np.diff(c.astype(np.int64))
    assert abs(m[0] / 2 ** 32 - (0.9 + 0.001)) < 1e-9 and np.all(m[1:] >= int(0.001 * 2 ** 32) - 1)


def test_pulse_injection_peaks_at_true_arrival(orc):
    """Noise-free pulse data injected at theta0 with arrival times t_c + dt_k(theta0): the window
    bin of the true time recovers <h0|h0>/2 (to the linear-interpolation error of the pulse peak),
    the peak sits there, and no sample exceeds <h0|h0>/2 (Cauchy-Schwarz)."""
    K, M, Nt = 3, 5, 64
    tens, pos = S.detector_arrays(K)
    rng = np.random.default_rng(17)
    for trial in range(4):
        theta0 = np.array([rng.uniform(0, 2 * np.pi), np.arcsin(rng.uniform(-1, 1)), rng.uniform(0, np.pi),
                           np.arccos(rng.uniform(-1, 1)), rng.uniform(0, 2 * np.pi), 250.0, 1.0 / S.FS])
        c0 = np.array([[(S.D_REF / theta0[5]) * orc.antenna(tens[k], *theta0[:3]) * orc.sylm(l, m, theta0[3], theta0[4])
                        for (l, m) in S.mode_list(M)] for k in range(K)])
        t0 = np.array([theta0[6] + orc.delay(pos[k], theta0[0], theta0[1]) for k in range(K)])
        point = S.make_point(1000 + trial, K, M, Nt, c_true=c0, t_true=t0, noise=0.0)
        lnL, _, A0 = orc.lnL_grid(point, theta0)
        j0 = Nt // 2
        assert 0.99 * A0 < lnL[j0] <= A0 * (1 + 1e-12)
        assert abs(int(np.argmax(lnL)) - j0) <= 1
        th = S.prior_samples(rng, 100)
        for n in range(th.shape[1]):
            assert np.all(orc.lnL_grid(point, th[:, n])[0] <= A0 * (1 + 1e-12))


# ------------------------------------------------------------------------------ rotated sky frame
def test_rotated_sky_frame_geometry_and_uniformity(orc):
    """The rotated network frame (R23): orthonormal and right-handed with the pole as third axis;
    a sample's rotated latitude is its angle to the pole; uniform tables give a uniform sky
    (the prior is rotation invariant); latitude +90 deg maps onto the pole direction."""
    sps = pytest.importorskip("scipy.stats")
    _, pos = S.detector_arrays(2)
    pole = pos[1] - pos[0]
    e1, e2, p = orc.sky_frame(pole)
    Mx = np.stack([e1, e2, p])
    np.testing.assert_allclose(Mx @ Mx.T, np.eye(3), atol=1e-14)
    np.testing.assert_allclose(np.cross(e1, e2), p, atol=1e-14)
    np.testing.assert_allclose(p, pole / np.linalg.norm(pole), atol=1e-15)
    lo, hi = [0.0, -1.0, 0.0, -1.0, 0.0, 100.0, -1e-3], [2 * np.pi, 1.0, np.pi, 1.0, 2 * np.pi, 1000.0, 1e-3]
    gmst = 0.7
    tabs = np.stack([orc.cdf_uniform() for _ in range(7)])
    smp = orc.make_sampler(lo, hi, [0] * 7, tabs, pole, gmst)
    th, lw, _ = orc.sample(smp, 99, 0, 0, 0, 20000)
    assert np.all(lw == 0.0)
    assert sps.kstest(np.sin(th[1]), "uniform", args=(-1, 2)).pvalue > 1e-3
    assert sps.kstest(th[0], "uniform", args=(0, 2 * np.pi)).pvalue > 1e-3
    # the rotated latitude (from the same words with no rotation) is the angle to the pole
    plain = orc.make_sampler(lo, hi, [0] * 7, tabs)
    thp, _, _ = orc.sample(plain, 99, 0, 0, 0, 2000)
    g = gmst - th[0, :2000]
    n = np.stack([np.cos(th[1, :2000]) * np.cos(g), -np.cos(th[1, :2000]) * np.sin(g), np.sin(th[1, :2000])])
    np.testing.assert_allclose(p @ n, np.sin(thp[1]), atol=1e-12)
    # longitude: angle around the pole from e1
    np.testing.assert_allclose(np.arctan2(e2 @ n, e1 @ n) % (2 * np.pi), thp[0] % (2 * np.pi), atol=1e-9)
    # a narrow band at latitude ~ +90 deg lands on the pole
    lo2 = list(lo)
    lo2[1] = 1 - 1e-9
    th2, _, _ = orc.sample(orc.make_sampler(lo2, hi, [0] * 7, tabs, pole, gmst), 5, 0, 0, 0, 50)
    g2 = gmst - th2[0]
    n2 = np.stack([np.cos(th2[1]) * np.cos(g2), -np.cos(th2[1]) * np.sin(g2), np.sin(th2[1])])
    assert np.all(p @ n2 > 1 - 1e-8)


def test_quv_structure_and_frequency_cut(orc):
    """U Hermitian and positive semi-definite, V symmetric (Eq. (eq:QUV)); Q at t = 0 is the plain
    sum; bins at or below f_low contribute nothing."""
    point, aux = _fd_setup(4)
    hf, psd, d_f, df = aux["hf"], aux["psd"], aux["d_f"], aux["df"]
    Q, U, V = orc.quv_from_modes(hf, psd, d_f, df, -1.0, 0.0, 4096.0, 3)
    for k in range(U.shape[0]):
        np.testing.assert_allclose(U[k], U[k].conj().T, atol=1e-12)
        assert np.linalg.eigvalsh(U[k]).min() > -1e-10
        np.testing.assert_allclose(V[k], V[k].T, atol=1e-12)
        for a in range(hf.shape[0]):
            assert abs(Q[k, a, 0] - 2 * df * np.sum(np.conj(hf[a]) * d_f[k] / psd[k])) < 1e-10
    f = np.fft.fftfreq(hf.shape[1], 1.0 / (hf.shape[1] * df))
    hcut = hf.copy()
    hcut[:, np.abs(f) <= 200.0] = 7.0  # junk below the cut must not matter
    Q2, U2, V2 = orc.quv_from_modes(hcut, psd, d_f, df, 200.0, 0.0, 4096.0, 3)
    Q3, U3, V3 = orc.quv_from_modes(hf, psd, d_f, df, 200.0, 0.0, 4096.0, 3)
    np.testing.assert_allclose(U2, U3, atol=1e-12)
    np.testing.assert_allclose(Q2, Q3, atol=1e-12)


def test_loud_injection_has_the_requested_strength(orc):
    """The loud points of the GPU tests: the injected template's <h0|h0>/2 (the oracle's quadratic
    term at theta0) equals rho2/2, and the window bin of the true arrival time recovers about that
    (the injection identity, up to the noise and the pulse's interpolation error)."""
    for rho2 in (1e2, 1e4):
        point, theta0 = orc.loud_point(S, S.SEED_BASE + 90, rho2)
        lnl, data, A = orc.lnL_grid(point, theta0)
        assert abs(A - rho2 / 2) < 1e-9 * rho2
        j0 = point.n_window // 2  # bin j is at t_c + (j - N_t/2)/f_s: theta0's own t_c is the true time
        assert abs(lnl.max() - rho2 / 2) < 0.05 * rho2 / 2 + 5.0
        assert abs(int(np.argmax(lnl)) - j0) <= 2


def test_nearest_sample_mode_brute_force(orc):
    """The oracle's nearest-sample mode (reading of the delay interpolation, exported as
    ILE_NEAREST) against a plain Python sum over the Q series with Python's own round-half-even,
    on a tiny point; where every detector's window start is an integer the nearest and linear
    modes agree."""
    point = S.make_point(S.SEED_BASE + 70, 2, 2, 8, spectrum="random")
    rng = np.random.default_rng(71)
    th = S.prior_samples(rng, 6)
    for n in range(th.shape[1]):
        t = th[:, n]
        lnl, data, A = orc.lnL_grid(point, t, nearest=True)
        ra, dec, psi, iota, phi, dist, tc = t
        y = np.array([orc.sylm(int(l), int(m), iota, phi) for l, m in point.lm])
        for j in range(point.n_window):
            want = 0.0
            for k in range(point.n_det):
                c = (point.d_ref / dist) * orc.antenna(point.det_tensor[k], ra, dec, psi) * y
                tau = tc + (j - point.n_window / 2) / point.fs + orc.delay(point.det_pos[k], ra, dec)
                i = round((tau - point.t_start) * point.fs)  # Python rounds half to even
                want += np.sum((np.conj(c) * point.Q[k, :, i]).real)
            assert abs(data[j] - want) < 1e-10 * max(1.0, abs(want)), (n, j)
            assert abs(lnl[j] - (want - A)) < 1e-10 * max(1.0, abs(want - A))
    # with a flat (time-independent) Q the choice of sample does not matter: the two modes agree
    flat = S.make_point(S.SEED_BASE + 72, 2, 2, 8, spectrum="random", pulse_sigma=None, noise=0.0)
    for n in range(th.shape[1]):
        a = orc.lnL_grid(flat, th[:, n], nearest=True)[0]
        b = orc.lnL_grid(flat, th[:, n])[0]
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
