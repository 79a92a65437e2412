"""FP64 CPU oracle for the ILE extrinsic-marginalisation hot path (arXiv:2210.07912).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
cpu_baseline / reference leg may import this package.  The CUDA library never loads it, and the
two share no code: the oracle is the plain C file ``ile_oracle.c`` next to this module, compiled
with gcc (``-O2 -ffp-contract=off -fopenmp``) and called through ctypes.

Every function cites the passage of the paper it follows in ``ile_oracle.c``.  Pins that tie the
oracle to something other than itself live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ile_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libile_oracle.so")
_lock = threading.Lock()
_lib = None

NBINS = 100
NDIM = 7


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libile_oracle.so`` (gcc, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Point(ctypes.Structure):
    _fields_ = [
        ("n_det", ctypes.c_int), ("n_modes", ctypes.c_int),
        ("lm", ctypes.c_void_p), ("det_tensor", ctypes.c_void_p), ("det_pos", ctypes.c_void_p),
        ("Q", ctypes.c_void_p), ("T_ext", ctypes.c_int), ("t_start", ctypes.c_double),
        ("fs", ctypes.c_double), ("U", ctypes.c_void_p), ("V", ctypes.c_void_p),
        ("n_window", ctypes.c_int), ("gmst", ctypes.c_double), ("d_ref", ctypes.c_double),
        ("nearest", ctypes.c_int),
    ]


GMM_MAX = 8


class _Gmm1(ctypes.Structure):
    _fields_ = [
        ("C", ctypes.c_int), ("w", ctypes.c_double * GMM_MAX), ("mu", ctypes.c_double * GMM_MAX),
        ("sigma", ctypes.c_double * GMM_MAX), ("n", ctypes.c_double),
    ]


class _Gmm2(ctypes.Structure):
    _fields_ = [
        ("C", ctypes.c_int), ("w", ctypes.c_double * GMM_MAX), ("mu", (ctypes.c_double * 2) * GMM_MAX),
        ("cov", (ctypes.c_double * 3) * GMM_MAX), ("n", ctypes.c_double),
    ]


class _Sampler(ctypes.Structure):
    _fields_ = [
        ("lo", ctypes.c_double * NDIM), ("hi", ctypes.c_double * NDIM),
        ("adaptive", ctypes.c_int * NDIM), ("cdf", ctypes.c_void_p),
        ("sky", ctypes.c_int), ("pole", ctypes.c_double * 3), ("gmst", ctypes.c_double),
        ("gmm", ctypes.c_int * NDIM), ("model", ctypes.c_void_p),
        ("pair", ctypes.c_int), ("pair_model", ctypes.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            lib.orc_frame.argtypes = [d, d, d, d, vp, vp, vp]
            lib.orc_antenna.argtypes = [vp, d, d, d, d, vp]
            lib.orc_delay.argtypes = [vp, d, d, d]
            lib.orc_delay.restype = d
            lib.orc_wigner_d.argtypes = [i, i, i, d]
            lib.orc_wigner_d.restype = d
            lib.orc_sylm.argtypes = [i, i, d, d, vp]
            lib.orc_lnL_grid.argtypes = [ctypes.POINTER(_Point), vp, vp, vp, vp]
            lib.orc_lnL_t.argtypes = [ctypes.POINTER(_Point), vp, ctypes.c_long, vp, i]
            lib.orc_mc_stats.argtypes = [vp, ctypes.c_long, vp]
            lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
            lib.orc_sample.argtypes = [ctypes.POINTER(_Sampler), ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_long, ctypes.c_long, vp, vp, vp, vp]
            lib.orc_norm_ppf.argtypes = [d]
            lib.orc_norm_ppf.restype = d
            lib.orc_gmm_cum.argtypes = [ctypes.POINTER(_Gmm1), vp]
            lib.orc_gmm_lnpdf.argtypes = [ctypes.POINTER(_Gmm1), d, d, d]
            lib.orc_gmm_lnpdf.restype = d
            lib.orc_gmm_init.argtypes = [ctypes.POINTER(_Gmm1), i, d, d]
            lib.orc_gmm_update.argtypes = [ctypes.POINTER(_Gmm1), vp, vp, ctypes.c_long, i, d, d]
            lib.orc_gmm_em_step.argtypes = [vp, vp, ctypes.c_long, ctypes.POINTER(_Gmm1), d, d]
            lib.orc_gmm_merge.argtypes = [ctypes.POINTER(_Gmm1), ctypes.POINTER(_Gmm1), d, ctypes.POINTER(_Gmm1)]
            lib.orc_hist.argtypes = [vp, vp, ctypes.c_long, vp]
            lib.orc_cdf_from_hist.argtypes = [vp, d, vp]
            lib.orc_cdf_uniform.argtypes = [vp]
            lib.orc_sky_frame.argtypes = [vp, vp, vp, vp]
            G2 = ctypes.POINTER(_Gmm2)
            lib.orc_bvn_rect.argtypes = [vp, vp, vp, vp]
            lib.orc_bvn_rect.restype = d
            lib.orc_gmm2_lnpdf.argtypes = [G2, vp, vp, vp]
            lib.orc_gmm2_lnpdf.restype = d
            lib.orc_gmm2_lnpdf_z.argtypes = [G2, vp, vp]
            lib.orc_gmm2_lnpdf_z.restype = d
            lib.orc_gmm2_masses.argtypes = [G2, vp, vp, vp]
            lib.orc_gmm2_em_step.argtypes = [vp, vp, vp, ctypes.c_long, G2, vp, vp]
            lib.orc_gmm2_merge.argtypes = [G2, G2, d, vp, vp, G2]
            lib.orc_gmm2_init.argtypes = [G2, i, vp, vp]
            lib.orc_gmm2_update.argtypes = [G2, vp, vp, vp, ctypes.c_long, i, vp, vp]
            lib.orc_pair_draw.argtypes = [G2, vp, vp, ctypes.c_uint32, vp, vp, vp, ctypes.POINTER(ctypes.c_int)]
            lib.orc_pair_draw.restype = i
            lib.orc_dmarg_lnF.argtypes = [d, d, d, d, d]
            lib.orc_dmarg_lnF.restype = d
            lib.orc_lnL_dmarg.argtypes = [ctypes.POINTER(_Point), vp, ctypes.c_long, d, d, vp]
            lib.orc_wigner_d_deriv.argtypes = [i, i, i, d]
            lib.orc_wigner_d_deriv.restype = d
            lib.orc_lnL_t_grad.argtypes = [ctypes.POINTER(_Point), vp, d, vp, vp, vp, vp, vp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _PointView:
    """Keeps the contiguous FP64 copies of a point alive while C reads them."""

    def __init__(self, p, nearest: bool = False):
        self.lm = np.ascontiguousarray(p.lm, dtype=np.int32)
        self.det_tensor = np.ascontiguousarray(p.det_tensor, dtype=np.float64)
        self.det_pos = np.ascontiguousarray(p.det_pos, dtype=np.float64)
        self.Q = np.ascontiguousarray(np.stack([p.Q.real, p.Q.imag], axis=-1), dtype=np.float64)
        self.U = np.ascontiguousarray(np.stack([p.U.real, p.U.imag], axis=-1), dtype=np.float64)
        self.V = np.ascontiguousarray(np.stack([p.V.real, p.V.imag], axis=-1), dtype=np.float64)
        K, M, T = p.Q.shape
        self.s = _Point(K, M, _ptr(self.lm).value, _ptr(self.det_tensor).value, _ptr(self.det_pos).value,
                        _ptr(self.Q).value, T, float(p.t_start), float(p.fs), _ptr(self.U).value,
                        _ptr(self.V).value, int(p.n_window), float(p.gmst), float(p.d_ref), int(bool(nearest)))


# ------------------------------------------------------------------------------------ S1 / S2
def frame(ra, dec, psi, gmst=0.0):
    X, Y, n = (np.zeros(3) for _ in range(3))
    _load().orc_frame(ra, dec, psi, gmst, _ptr(X), _ptr(Y), _ptr(n))
    return X, Y, n


def antenna(D, ra, dec, psi, gmst=0.0) -> complex:
    D = np.ascontiguousarray(D, dtype=np.float64)
    out = np.zeros(2)
    _load().orc_antenna(_ptr(D), ra, dec, psi, gmst, _ptr(out))
    return complex(out[0], out[1])


def delay(r, ra, dec, gmst=0.0) -> float:
    r = np.ascontiguousarray(r, dtype=np.float64)
    return _load().orc_delay(_ptr(r), ra, dec, gmst)


def wigner_d(l, m1, m2, beta) -> float:
    return _load().orc_wigner_d(l, m1, m2, beta)


def wigner_d_deriv(l, m1, m2, beta) -> float:
    """d/dbeta of d^l_{m1,m2}(beta)."""
    return _load().orc_wigner_d_deriv(l, m1, m2, beta)


def sylm(l, m, iota, phi) -> complex:
    out = np.zeros(2)
    _load().orc_sylm(l, m, iota, phi, _ptr(out))
    return complex(out[0], out[1])


# ------------------------------------------------------------------------------------ S3-S5
class RangeError(ValueError):
    pass


def lnL_grid(point, theta, nearest: bool = False):
    """lnL(j) for j < N_t of one sample theta (7,), plus the data term and A = <h|h>/2.
    nearest: Q at the nearest sample instead of the linear interpolation."""
    pv = _PointView(point, nearest)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    lnL = np.zeros(point.n_window)
    data = np.zeros(point.n_window)
    A = np.zeros(1)
    st = _load().orc_lnL_grid(ctypes.byref(pv.s), _ptr(th), _ptr(lnL), _ptr(data), _ptr(A))
    if st == 3:
        raise RangeError("interpolation index outside [0, T_ext-1]")
    if st != 0:
        raise ValueError(f"oracle status {st}")
    return lnL, data, float(A[0])


def lnL_t(point, samples, nthreads: int = 0, nearest: bool = False):
    """Time-marginalised lnL of every sample; samples is SoA (7, N).  nearest: Q at the nearest
    sample instead of the linear interpolation."""
    pv = _PointView(point, nearest)
    s = np.ascontiguousarray(samples, dtype=np.float64)
    N = s.shape[1]
    out = np.zeros(N)
    st = _load().orc_lnL_t(ctypes.byref(pv.s), _ptr(s), N, _ptr(out), int(nthreads))
    if st == 3:
        raise RangeError("interpolation index outside [0, T_ext-1]")
    if st != 0:
        raise ValueError(f"oracle status {st}")
    return out


def lnL_t_grad(point, samples, g=None):
    """Analytic gradient of lnL_t for samples (7, N) times upstream weights g (N,) (default 1):
    returns (lnL_t (N,), g_theta (7, N), g_Q (K, M, T, 2), g_U (K, M, M, 2), g_V (K, M, M, 2)), the
    Q/U/V gradients summed over the samples and taken entry by entry as independent reals."""
    pv = _PointView(point)
    s = np.ascontiguousarray(samples, dtype=np.float64)
    N = s.shape[1]
    g = np.ones(N) if g is None else np.asarray(g, np.float64)
    K, M, T = point.Q.shape
    gQ = np.zeros((K, M, T, 2))
    gU = np.zeros((K, M, M, 2))
    gV = np.zeros((K, M, M, 2))
    gth = np.zeros((7, N))
    out = np.zeros(N)
    lib = _load()
    for n in range(N):
        th = np.ascontiguousarray(s[:, n])
        gt = np.zeros(7)
        lt = np.zeros(1)
        st = lib.orc_lnL_t_grad(ctypes.byref(pv.s), _ptr(th), float(g[n]), _ptr(gt), _ptr(gQ), _ptr(gU), _ptr(gV),
                                _ptr(lt))
        if st == 3:
            raise RangeError("interpolation index outside [0, T_ext-1]")
        gth[:, n] = gt
        out[n] = lt[0]
    return out, gth, gQ, gU, gV


def dmarg_lnF(a, b, d_min, d_max, d_ref):
    """ln int p(D) exp(a x - b x^2) dD, x = d_ref / D, p prop. to D^2 on [d_min, d_max]."""
    return _load().orc_dmarg_lnF(float(a), float(b), float(d_min), float(d_max), float(d_ref))


def lnL_dmarg(point, samples, d_min, d_max):
    """Distance- and time-marginalised lnL of every sample (the samples' D is ignored)."""
    pv = _PointView(point)
    s = np.ascontiguousarray(samples, dtype=np.float64)
    N = s.shape[1]
    out = np.zeros(N)
    st = _load().orc_lnL_dmarg(ctypes.byref(pv.s), _ptr(s), N, float(d_min), float(d_max), _ptr(out))
    if st == 3:
        raise RangeError("interpolation index outside [0, T_ext-1]")
    if st != 0:
        raise ValueError(f"oracle status {st}")
    return out


def quv_from_modes(hf, psd, d_f, df, f_low, t_start, fs, T_ext):
    """Eq. (eq:QUV) written out in FP64 for discrete two-sided frequency series in FFT order:
    Q_k,a(t) = 2 df sum_{|f|>f_low} e^{2 pi i f t} conj(h_a(f)) d_k(f) / S_k(f) at
    t = t_start + i / fs (i < T_ext); U_k,ab = <h_a|h_b>_k; V_k,ab = <h_a^*|h_b>_k, where the
    Fourier transform of conj(h_a(t)) is conj(h_a(-f)).  Returns complex Q (K, M, T_ext), U, V (K, M, M)."""
    hf = np.asarray(hf, complex)
    d_f = np.asarray(d_f, complex)
    psd = np.asarray(psd, float)
    M, L = hf.shape
    K = d_f.shape[0]
    f = np.fft.fftfreq(L, 1.0 / (L * df))
    keep = np.abs(f) > f_low
    hstar = np.conj(hf[:, (-np.arange(L)) % L])
    U = np.zeros((K, M, M), complex)
    V = np.zeros((K, M, M), complex)
    Q = np.zeros((K, M, T_ext), complex)
    times = t_start + np.arange(T_ext) / fs
    phase = np.exp(2j * np.pi * np.outer(times, f[keep]))  # (T_ext, bins kept)
    for k in range(K):
        w = 2.0 * df / psd[k]
        for a in range(M):
            for b in range(M):
                U[k, a, b] = np.sum((np.conj(hf[a]) * hf[b] * w)[keep])
                V[k, a, b] = np.sum((np.conj(hstar[a]) * hf[b] * w)[keep])
            Q[k, a] = phase @ (np.conj(hf[a]) * d_f[k] * w)[keep]
    return Q, U, V


# ------------------------------------------------------------------------------------ S6
def mc_stats(lnw):
    """Eq. (eq:lnL:MonteCarlo) in log space: dict(ln_I, sigma_ln, n_eff, ess, m, s1, s2)."""
    lnw = np.ascontiguousarray(lnw, dtype=np.float64)
    out = np.zeros(7)
    _load().orc_mc_stats(_ptr(lnw), lnw.size, _ptr(out))
    return dict(ln_I=out[0], sigma_ln=out[1], n_eff=out[2], ess=out[3], m=out[4], s1=out[5], s2=out[6])


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


# ------------------------------------------------------------------------------------ mixture sampler
def _gmm_struct(m):
    g = _Gmm1()
    C = len(m["w"])
    g.C = C
    for c in range(C):
        g.w[c], g.mu[c], g.sigma[c] = float(m["w"][c]), float(m["mu"][c]), float(m["sigma"][c])
    g.n = float(m.get("n", 0.0))
    return g


def _gmm_dict(g):
    C = g.C
    return dict(w=np.array(g.w[:C]), mu=np.array(g.mu[:C]), sigma=np.array(g.sigma[:C]), n=float(g.n))


def gmm_init(C: int, lo: float, hi: float):
    g = _Gmm1()
    _load().orc_gmm_init(ctypes.byref(g), int(C), float(lo), float(hi))
    return _gmm_dict(g)


def gmm_lnpdf(m, lo: float, hi: float, u: float) -> float:
    g = _gmm_struct(m)
    return _load().orc_gmm_lnpdf(ctypes.byref(g), float(lo), float(hi), float(u))


def gmm_cum(m):
    g = _gmm_struct(m)
    cw = np.zeros(GMM_MAX + 1, dtype=np.uint64)
    _load().orc_gmm_cum(ctypes.byref(g), _ptr(cw))
    return cw[: g.C + 1]


def gmm_update(m, u, w, iters: int, lo: float, hi: float):
    """EM on the batch (u, weights w) from the current model, then the online merge."""
    g = _gmm_struct(m)
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    _load().orc_gmm_update(ctypes.byref(g), _ptr(u), _ptr(w), u.size, int(iters), float(lo), float(hi))
    return _gmm_dict(g)


def gmm_em_step(m, u, w, lo: float, hi: float):
    g = _gmm_struct(m)
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    _load().orc_gmm_em_step(_ptr(u), _ptr(w), u.size, ctypes.byref(g), float(lo), float(hi))
    return _gmm_dict(g)


def gmm_merge(cur, bat, M: float):
    a, b, out = _gmm_struct(cur), _gmm_struct(bat), _Gmm1()
    _load().orc_gmm_merge(ctypes.byref(a), ctypes.byref(b), float(M), ctypes.byref(out))
    return _gmm_dict(out)


# ------------------------------------------------------------------------------------ correlated sky pair
def _gmm2_struct(m):
    g = _Gmm2()
    C = len(m["w"])
    g.C = C
    for c in range(C):
        g.w[c] = float(m["w"][c])
        for j in range(2):
            g.mu[c][j] = float(m["mu"][c][j])
        for j in range(3):
            g.cov[c][j] = float(m["cov"][c][j])
    g.n = float(m.get("n", 0.0))
    return g


def _gmm2_dict(g):
    C = g.C
    return dict(w=np.array(g.w[:C]), mu=np.array([[g.mu[c][0], g.mu[c][1]] for c in range(C)]),
                cov=np.array([[g.cov[c][0], g.cov[c][1], g.cov[c][2]] for c in range(C)]), n=float(g.n))


def _v2(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def bvn_rect(mu, cov, lo, hi) -> float:
    """Mass of the rectangle [lo0, hi0] x [lo1, hi1] under N(mu, [[cov0, cov1], [cov1, cov2]])."""
    a, b, c, e = _v2(mu), _v2(cov), _v2(lo), _v2(hi)
    return _load().orc_bvn_rect(_ptr(a), _ptr(b), _ptr(c), _ptr(e))


def gmm2_init(C: int, lo, hi):
    g = _Gmm2()
    a, b = _v2(lo), _v2(hi)
    _load().orc_gmm2_init(ctypes.byref(g), int(C), _ptr(a), _ptr(b))
    return _gmm2_dict(g)


def gmm2_masses(m, lo, hi):
    """Each component's mass inside the rectangle."""
    g = _gmm2_struct(m)
    a, b = _v2(lo), _v2(hi)
    Z = np.zeros(GMM_MAX)
    _load().orc_gmm2_masses(ctypes.byref(g), _ptr(a), _ptr(b), _ptr(Z))
    return Z[: g.C]


def gmm2_lnpdf(m, lo, hi, x, Z=None) -> float:
    """ln of the truncated pair density at x (Z: the masses from gmm2_masses, else computed)."""
    g = _gmm2_struct(m)
    if Z is None:
        a, b, c = _v2(lo), _v2(hi), _v2(x)
        return _load().orc_gmm2_lnpdf(ctypes.byref(g), _ptr(a), _ptr(b), _ptr(c))
    z = np.zeros(GMM_MAX)
    z[: len(Z)] = Z
    c = _v2(x)
    return _load().orc_gmm2_lnpdf_z(ctypes.byref(g), _ptr(z), _ptr(c))


def gmm2_em_step(m, u0, u1, w, lo, hi):
    g = _gmm2_struct(m)
    x0, x1, ww, a, b = _v2(u0), _v2(u1), _v2(w), _v2(lo), _v2(hi)
    _load().orc_gmm2_em_step(_ptr(x0), _ptr(x1), _ptr(ww), x0.size, ctypes.byref(g), _ptr(a), _ptr(b))
    return _gmm2_dict(g)


def gmm2_merge(cur, bat, M: float, lo, hi):
    a, b, out = _gmm2_struct(cur), _gmm2_struct(bat), _Gmm2()
    l, h = _v2(lo), _v2(hi)
    _load().orc_gmm2_merge(ctypes.byref(a), ctypes.byref(b), float(M), _ptr(l), _ptr(h), ctypes.byref(out))
    return _gmm2_dict(out)


def gmm2_update(m, u0, u1, w, iters: int, lo, hi):
    """EM on the batch (points (u0, u1), weights w) from the current pair model, then the merge."""
    g = _gmm2_struct(m)
    x0, x1, ww, a, b = _v2(u0), _v2(u1), _v2(w), _v2(lo), _v2(hi)
    _load().orc_gmm2_update(ctypes.byref(g), _ptr(x0), _ptr(x1), _ptr(ww), x0.size, int(iters), _ptr(a), _ptr(b))
    return _gmm2_dict(g)


def pair_draw(m, lo, hi, a_word: int, ctr0, key):
    """One draw of the pair (see orc_pair_draw): returns (x (2,), component, attempts)."""
    g = _gmm2_struct(m)
    l, h = _v2(lo), _v2(hi)
    c0 = np.ascontiguousarray(ctr0, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    x = np.zeros(2)
    comp = ctypes.c_int()
    t = _load().orc_pair_draw(ctypes.byref(g), _ptr(l), _ptr(h), int(a_word), _ptr(c0), _ptr(k), _ptr(x),
                              ctypes.byref(comp))
    return x, comp.value, t


def norm_ppf(p: float) -> float:
    return _load().orc_norm_ppf(float(p))


def make_sampler(lo, hi, adaptive, cdf, sky_pole=None, gmst=0.0, gmm=None, pair=None):
    """sky_pole: pole of the rotated network sky frame (variables 0, 1 in that frame), or None.
    gmm: None or a list of 7 entries, each None (histogram / prior) or a mixture model dict
    (w, mu, sigma, n) for an adaptive dimension drawn from its Gaussian mixture.
    pair: None or a pair model dict (w, mu (C,2), cov (C,3), n): variables 0 and 1 drawn together
    from the correlated mixture."""
    cdf = np.ascontiguousarray(cdf, dtype=np.uint64).reshape(NDIM, NBINS + 1)
    pole = (0.0, 0.0, 0.0) if sky_pole is None else tuple(float(x) for x in sky_pole)
    models = (_Gmm1 * NDIM)()
    flags = [0] * NDIM
    if gmm is not None:
        for d in range(NDIM):
            if gmm[d] is not None:
                models[d] = _gmm_struct(gmm[d])
                flags[d] = 1
    s = _Sampler((ctypes.c_double * NDIM)(*lo), (ctypes.c_double * NDIM)(*hi),
                 (ctypes.c_int * NDIM)(*[int(a) for a in adaptive]), _ptr(cdf).value, 0 if sky_pole is None else 1,
                 (ctypes.c_double * 3)(*pole), float(gmst), (ctypes.c_int * NDIM)(*flags),
                 ctypes.cast(models, ctypes.c_void_p).value)
    pm = None
    if pair is not None:
        pm = _gmm2_struct(pair)
        s.pair = 1
        s.pair_model = ctypes.cast(ctypes.pointer(pm), ctypes.c_void_p).value
    s._keep = (cdf, models, pm)
    return s


def sky_frame(pole):
    e1, e2, p = np.zeros(3), np.zeros(3), np.zeros(3)
    pole = np.ascontiguousarray(pole, dtype=np.float64)
    _load().orc_sky_frame(_ptr(pole), _ptr(e1), _ptr(e2), _ptr(p))
    return e1, e2, p


def sample(sampler, seed: int, it: int, point: int, n0: int, N: int, with_u: bool = False):
    """Device-sampler definition: returns theta (7,N), ln p - ln p_s (N,), bins (7,N) uint8
    (the mixture component for a mixture dimension), and with with_u the sampling variables u (7,N)."""
    theta = np.zeros((NDIM, N))
    lw = np.zeros(N)
    bins = np.zeros((NDIM, N), dtype=np.uint8)
    u = np.zeros((NDIM, N))
    _load().orc_sample(ctypes.byref(sampler), seed, it, point, n0, N, _ptr(theta), _ptr(lw), _ptr(bins), _ptr(u))
    return (theta, lw, bins, u) if with_u else (theta, lw, bins)


def hist(lnw, bins):
    lnw = np.ascontiguousarray(lnw, dtype=np.float64)
    b = np.ascontiguousarray(bins, dtype=np.uint8)
    h = np.zeros(NBINS)
    _load().orc_hist(_ptr(lnw), _ptr(b), lnw.size, _ptr(h))
    return h


def cdf_from_hist(h, eps: float = 0.1):
    h = np.ascontiguousarray(h, dtype=np.float64)
    cdf = np.zeros(NBINS + 1, dtype=np.uint64)
    _load().orc_cdf_from_hist(_ptr(h), eps, _ptr(cdf))
    return cdf


def cdf_uniform():
    cdf = np.zeros(NBINS + 1, dtype=np.uint64)
    _load().orc_cdf_uniform(_ptr(cdf))
    return cdf


# ------------------------------------------------------------------------------------ S0-S6 loop
def adapt_run(point, seed: int, N: int, n_iter: int, adapt_mask: int, eps: float, lo, hi, point_id: int = 0,
              nthreads: int = 0, cdf0=None, iter0: int = 0, sky_pole=None, gmm_mask: int = 0,
              gmm_components: int = 3, gmm_em_iters: int = 8, gmm0=None, gmm_pair: bool = False, pair0=None):
    """Adaptive-Cartesian integration in the order of Sec. "GPU-accelerated Monte Carlo integration":
    for each iteration draw N samples from the separable sampling prior, evaluate lnL_t, accumulate
    the Monte Carlo sums of Eq. (eq:lnL:MonteCarlo) (pooled over iterations, each sample weighted by
    the p_s it was drawn from) and refit each adaptive dimension's 100-bin histogram.
    Adaptive dimensions in gmm_mask are drawn from a truncated Gaussian mixture instead
    (Sec. "Adaptive sampling with gaussian mixture models"), refit each iteration by gmm_update;
    with gmm_pair the sky pair (variables 0 and 1) is drawn from one correlated mixture, refit by
    gmm2_update.
    Returns the pooled estimate, the per-iteration estimates, the final tables and mixtures, and the
    last iteration's samples."""
    adaptive = [(adapt_mask >> d) & 1 for d in range(NDIM)]
    gmm = [None] * NDIM
    for d in range(NDIM):
        if adaptive[d] and (gmm_mask >> d) & 1:
            gmm[d] = dict(gmm0[d]) if gmm0 is not None else gmm_init(gmm_components, lo[d], hi[d])
    plo, phi_ = [lo[0], lo[1]], [hi[0], hi[1]]
    pair = None
    if gmm_pair:
        pair = dict(pair0) if pair0 is not None else gmm2_init(gmm_components, plo, phi_)
    cdf = np.zeros((NDIM, NBINS + 1), np.uint64)
    for d in range(NDIM):
        cdf[d] = cdf_uniform() if cdf0 is None else cdf0[d]
    lnw_all = []
    iters = []
    last = None
    for it in range(iter0, iter0 + n_iter):
        smp = make_sampler(lo, hi, adaptive, cdf, sky_pole, point.gmst, gmm, pair)
        theta, lwp, bins, u = sample(smp, seed, it, point_id, 0, N, with_u=True)
        lnl = lnL_t(point, theta, nthreads)
        lnw = lnl + lwp
        st = mc_stats(lnw)
        iters.append(st)
        lnw_all.append(lnw)
        hists = np.zeros((NDIM, NBINS))
        gmm_before = [None if g is None else dict(g) for g in gmm]
        pair_before = None if pair is None else dict(pair)
        if pair is not None:
            pair = gmm2_update(pair, u[0], u[1], np.exp(lnw - lnw.max()), gmm_em_iters, plo, phi_)
        for d in range(NDIM):
            if pair is not None and d < 2:
                continue
            if gmm[d] is not None:
                gmm[d] = gmm_update(gmm[d], u[d], np.exp(lnw - lnw.max()), gmm_em_iters, lo[d], hi[d])
            elif adaptive[d]:
                hists[d] = hist(lnw, bins[d])
                cdf[d] = cdf_from_hist(hists[d], eps)
        last = dict(theta=theta, lnw_prior=lwp, bins=bins, lnL=lnl, hist=hists, u=u, gmm=gmm_before,
                    pair=pair_before)
    pooled = mc_stats(np.concatenate(lnw_all))
    return dict(pooled=pooled, iters=iters, cdf=cdf, last=last, gmm=gmm, pair=pair)


# ------------------------------------------------------------------------------------ loud injections
def injection_coeffs(point, theta0):
    """True coefficients c0_k,lm = (D_ref/D) F_k Y_lm and arrival times t0_k = t_c + dt_k of the
    extrinsic sample theta0 (7,) for the detectors and modes of `point` (Eq. (eq:loglikelihood):
    the coefficients of the likelihood's h_k at theta0)."""
    K, M = point.n_det, point.n_modes
    ra, dec, psi, iota, phi, dist, tc = (float(x) for x in theta0)
    c0 = np.array([[(point.d_ref / dist) * antenna(point.det_tensor[k], ra, dec, psi, point.gmst) *
                    sylm(int(l), int(m), iota, phi) for (l, m) in point.lm] for k in range(K)])
    t0 = np.array([tc + delay(point.det_pos[k], ra, dec, point.gmst) for k in range(K)])
    return c0, t0


def loud_point(S, seed: int, rho2: float, n_det: int = 3, n_modes: int = 21, n_window: int = 512,
               spectrum: str = "decay", theta0=None):
    """A loud intrinsic point: a pulse injected at theta0 with <h0|h0> = rho2 (so the data term of
    samples near theta0 is about rho2 and lnL_t about rho2/2), the U and V of the synthetic
    recipe scaled up until the injection has that strength (App. "Choices for finite-precision
    floating point arithmetic and overflow" discusses SNRs rho ~ 35 and beyond).  S is the
    synthetic-input module.  Returns (point, theta0)."""
    if theta0 is None:
        theta0 = np.array([1.3, 0.35, 0.8, 0.6, 2.2, 400.0, 0.5 / S.FS])
    theta0 = np.asarray(theta0, float)
    probe = S.make_point(seed, n_det, n_modes, n_window, spectrum=spectrum, noise=0.0, pulse_sigma=None)
    c0, t0 = injection_coeffs(probe, theta0)
    _, _, A0 = lnL_grid(probe, theta0)          # A = <h|h>/2 of theta0 at unit scale
    scale = rho2 / (2.0 * A0)
    point = S.make_point(seed, n_det, n_modes, n_window, spectrum=spectrum, c_true=c0, t_true=t0, uv_scale=scale)
    return point, theta0


def loud_samples(S, rng, theta0, n_near: int, n_prior: int, spread: float = 1.0):
    """Samples for a loud point: n_near Gaussian perturbations of theta0 (the region that holds the
    posterior mass and the largest |lnL_t|) followed by n_prior draws from the extrinsic prior."""
    sd = spread * np.array([0.02, 0.02, 0.05, 0.05, 0.05, 0.0, 0.2 / S.FS])
    near = theta0[:, None] + sd[:, None] * rng.normal(size=(7, n_near))
    near[5] = theta0[5] * np.exp(0.05 * spread * rng.normal(size=n_near))
    near[0] = np.mod(near[0], 2 * np.pi)
    near[1] = np.clip(near[1], -1.5, 1.5)
    near[6] = np.clip(near[6], -3.5 / S.FS, 3.5 / S.FS)
    return np.concatenate([near, S.prior_samples(rng, n_prior)], axis=1)
