"""Seeded synthetic inputs for the ILE hot path.

This module only draws numbers: detector descriptions, the U/V/Q inner-product arrays of one
intrinsic point, and extrinsic samples from the prior.  It holds none of the likelihood's
arithmetic (no antenna pattern, harmonic, delay, contraction or log-sum-exp), so that the CUDA
library and the FP64 oracle can both be fed from it without sharing a step of the method.

Recipe (the paper's production ILE workloads stand in for real strain, which is not used):
  * detectors H1, L1, V1 (and K1): vertex positions and arm directions, Earth-fixed frame;
    response tensor D = (u u^T - v v^T)/2 for unit arm vectors u, v;
  * sample rate 4096 Hz, time window N_t bins, extended series T_ext bins starting at
    -T_ext/(2 f_s): T_ext = N_t + 2 (ceil(max|r_k|/c f_s + T_c f_s) + 1) rounded up to 32;
  * modes: prefix of the canonical order (l ascending, |m| descending, +m before -m);
  * U_k: "random" = A A^H with E|A_ij|^2 = 100/M, or "decay" = W diag(100 2^-i) W^H with W a
    Haar-random unitary; V_k = R^T K R with R = U_k^{1/2}, K = (B B^T)/(2 ||B B^T||_2), which keeps
    <h|h> > 0 for every coefficient vector;
  * Q_k(t) = 1/2 (U_k c0_k + conj(V_k) conj(c0_k)) g_k(t) + noise, with g_k a Gaussian pulse
    (sigma 2 ms) centred at the true arrival time t0_k and unit complex noise (E|n|^2 = 1).
    The true coefficients c0_k and arrival times t0_k are inputs; without them they are drawn at
    random (complex Gaussian coefficients, arrival times spread over the light-travel range);
  * extrinsic samples from the prior: uniform sky, psi in [0, pi), cos(iota) in [-1, 1],
    phi in [0, 2 pi), D prop. to D^2 on [100, 1000] Mpc, t_c uniform in [-T_c, T_c], T_c = 4/f_s.
Draw order: detectors -> U -> V -> true signal -> Q noise -> samples; numpy PCG64 seeded with
2210079120 + config index.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2210079120
C_SI = 299792458.0
FS = 4096.0
D_REF = 100.0
D_MIN, D_MAX = 100.0, 1000.0

# Vertex (m) and unit arm directions (x arm, y arm), Earth-fixed; public geodetic data.
DETECTORS = {
    "H1": ((-2.16141492636e6, -3.83469517889e6, 4.60035022664e6),
           (-0.22389266154, 0.79983062746, 0.55690487831),
           (-0.91397818574, 0.02609403989, -0.40492342125)),
    "L1": ((-7.42760447238e4, -5.49628371971e6, 3.22425701744e6),
           (-0.95457412153, -0.14158077340, -0.26218911324),
           (0.29774156894, -0.48791033647, -0.82054461286)),
    "V1": ((4.54637409900e6, 8.42989697626e5, 4.37857696241e6),
           (-0.70045821479, 0.20848948619, 0.68256166277),
           (-0.05379255368, -0.96908180549, 0.24080451708)),
    "K1": ((-3.77772e6, 3.48419e6, 3.76502e6),
           (-0.3759040, -0.8361583, 0.3994189),
           (0.7164378, 0.01114076, 0.6975620)),
}
NETWORK = ("H1", "L1", "V1", "K1")

# Canonical mode order: l ascending, |m| descending, +m before -m.
ALL_MODES = [(l, s * am) for l in (2, 3, 4) for am in range(l, -1, -1) for s in ((1, -1) if am else (1,))]


def mode_list(n_modes: int):
    """First n_modes of the canonical order: 2 -> (2,+-2); 5 -> l=2; 9 -> +(3,+-3),(3,+-2); 21 -> l<=4."""
    if not 1 <= n_modes <= len(ALL_MODES):
        raise ValueError(f"n_modes must be in [1, {len(ALL_MODES)}]")
    return np.array(ALL_MODES[:n_modes], dtype=np.int32)


def detector_arrays(n_det: int):
    """Response tensors (K,3,3) and vertex positions (K,3) of the first n_det network detectors."""
    tens, pos = [], []
    for name in NETWORK[:n_det]:
        r, u, v = (np.array(x, dtype=np.float64) for x in DETECTORS[name])
        u /= np.linalg.norm(u)
        v /= np.linalg.norm(v)
        tens.append(0.5 * (np.outer(u, u) - np.outer(v, v)))
        pos.append(r)
    return np.array(tens), np.array(pos)


def t_ext_for(n_window: int, det_pos, fs: float = FS, tc_max: float | None = None) -> int:
    if tc_max is None:
        tc_max = 4.0 / fs
    max_delay_bins = max(np.linalg.norm(r) for r in det_pos) / C_SI * fs
    half = math.ceil(max_delay_bins + tc_max * fs) + 1
    return int(32 * math.ceil((n_window + 2 * half) / 32))


@dataclasses.dataclass
class Point:
    """Inputs of one intrinsic point (what ile_set_data receives)."""
    lm: np.ndarray            # (M, 2) int32
    det_tensor: np.ndarray    # (K, 3, 3)
    det_pos: np.ndarray       # (K, 3) metres
    Q: np.ndarray             # (K, M, T_ext) complex128
    U: np.ndarray             # (K, M, M) complex128, Hermitian
    V: np.ndarray             # (K, M, M) complex128, symmetric
    t_start: float
    fs: float
    n_window: int
    gmst: float = 0.0
    d_ref: float = D_REF
    tc_max: float = 4.0 / FS

    @property
    def n_det(self):
        return self.Q.shape[0]

    @property
    def n_modes(self):
        return self.Q.shape[1]

    @property
    def T_ext(self):
        return self.Q.shape[2]


def _cgauss(rng, shape, var=1.0):
    s = math.sqrt(var / 2.0)
    return rng.normal(0.0, s, shape) + 1j * rng.normal(0.0, s, shape)


def _haar_unitary(rng, M):
    Z = _cgauss(rng, (M, M))
    Qm, R = np.linalg.qr(Z)
    d = np.diag(R)
    return Qm * (d / np.abs(d))


def _sqrt_psd(U):
    w, W = np.linalg.eigh(U)
    return (W * np.sqrt(np.clip(w, 0.0, None))) @ W.conj().T


def draw_UV(rng, n_det, n_modes, spectrum="random", scale=1.0):
    U = np.zeros((n_det, n_modes, n_modes), complex)
    V = np.zeros_like(U)
    for k in range(n_det):
        if spectrum == "random":
            A = _cgauss(rng, (n_modes, n_modes), 100.0 / n_modes)
            U[k] = A @ A.conj().T
        elif spectrum == "decay":
            W = _haar_unitary(rng, n_modes)
            U[k] = (W * (100.0 * 2.0 ** -np.arange(n_modes))) @ W.conj().T
        else:
            raise ValueError(spectrum)
        U[k] = 0.5 * (U[k] + U[k].conj().T)
    for k in range(n_det):
        B = _cgauss(rng, (n_modes, n_modes))
        Km = B @ B.T
        Km = 0.5 * Km / np.linalg.norm(Km, 2)
        R = _sqrt_psd(U[k])
        V[k] = R.T @ Km @ R
        V[k] = 0.5 * (V[k] + V[k].T)
    return scale * U, scale * V


def make_point(seed: int, n_det: int, n_modes: int, n_window: int, *, fs: float = FS,
               spectrum: str = "random", c_true=None, t_true=None, noise: float = 1.0,
               pulse_sigma: float | None = 2e-3, gmst: float = 0.0, uv_scale: float = 1.0) -> Point:
    """One synthetic intrinsic point.

    c_true: (K, M) complex true coefficients (F_k Y_lm D_ref/D at the injected sample), or None
    to draw them; t_true: (K,) true arrival times at each detector (s), or None to draw them.
    pulse_sigma=None gives a flat profile (g = 1).  uv_scale multiplies U and V (and with them
    the signal part of Q): a louder detector network, <h|h> and the data term grow in proportion.
    """
    rng = np.random.default_rng(seed)
    tens, pos = detector_arrays(n_det)
    lm = mode_list(n_modes)
    T_ext = t_ext_for(n_window, pos, fs)
    t_start = -(T_ext // 2) / fs
    U, V = draw_UV(rng, n_det, n_modes, spectrum, uv_scale)
    if c_true is None:
        amp = rng.normal(0.0, 0.5, n_det) + 1j * rng.normal(0.0, 0.5, n_det)
        y = _cgauss(rng, n_modes, 0.3)
        c_true = amp[:, None] * y[None, :]
    c_true = np.asarray(c_true, complex).reshape(n_det, n_modes)
    if t_true is None:
        span = max(np.linalg.norm(r) for r in pos) / C_SI
        t_true = rng.uniform(-span, span, n_det)
    t_true = np.asarray(t_true, float).reshape(n_det)
    t = t_start + np.arange(T_ext) / fs
    Q = np.zeros((n_det, n_modes, T_ext), complex)
    for k in range(n_det):
        peak = 0.5 * (U[k] @ c_true[k] + V[k].conj() @ c_true[k].conj())
        g = np.ones(T_ext) if pulse_sigma is None else np.exp(-0.5 * ((t - t_true[k]) / pulse_sigma) ** 2)
        Q[k] = peak[:, None] * g[None, :]
    if noise:
        Q += noise * _cgauss(rng, Q.shape)
    return Point(lm=lm, det_tensor=tens, det_pos=pos, Q=Q, U=U, V=V, t_start=t_start, fs=fs,
                 n_window=n_window, gmst=gmst)


def prior_samples(rng, N: int, fs: float = FS, tc_max: float | None = None):
    """Extrinsic samples from the prior, SoA (7, N): ra, dec, psi, iota, phi, D_Mpc, tc_s."""
    if tc_max is None:
        tc_max = 4.0 / fs
    ra = rng.uniform(0.0, 2 * math.pi, N)
    dec = np.arcsin(rng.uniform(-1.0, 1.0, N))
    psi = rng.uniform(0.0, math.pi, N)
    iota = np.arccos(rng.uniform(-1.0, 1.0, N))
    phi = rng.uniform(0.0, 2 * math.pi, N)
    u = rng.uniform(0.0, 1.0, N)
    dist = np.cbrt(D_MIN ** 3 + u * (D_MAX ** 3 - D_MIN ** 3))
    tc = rng.uniform(-tc_max, tc_max, N)
    return np.stack([ra, dec, psi, iota, phi, dist, tc])


# Synthetic workloads, named by their shape (the sizes of the paper's production ILE runs: 3
# detectors at 4096 Hz, modes up to l = 4; plus a small two-detector case the oracle evaluates
# in full).  "seed" offsets SEED_BASE for the point and its samples.
SMALL = "hl_m2_nt256"      # H1, L1; modes (2, +-2); N_t = 256; 2^14 samples
FULL = "hlv_m21_nt512"     # H1, L1, V1; 21 modes; N_t = 512; 2^20 samples
GRAD = "hlv_m21_nt512_g"   # the same shape with 2^18 samples, for the adjoint
WORKLOADS = {
    SMALL: dict(n_det=2, n_modes=2, n_window=256, n_samples=1 << 14, spectrum="random", seed=0),
    FULL: dict(n_det=3, n_modes=21, n_window=512, n_samples=1 << 20, spectrum="decay", seed=1),
    GRAD: dict(n_det=3, n_modes=21, n_window=512, n_samples=1 << 18, spectrum="decay", seed=4),
}


def workload_point(name: str, **kw) -> Point:
    c = WORKLOADS[name]
    return make_point(SEED_BASE + c["seed"], c["n_det"], c["n_modes"], c["n_window"], spectrum=c["spectrum"], **kw)


def workload_samples(name: str, N: int | None = None):
    c = WORKLOADS[name]
    rng = np.random.default_rng([SEED_BASE + c["seed"], 1])
    return prior_samples(rng, c["n_samples"] if N is None else N)


def batch_descs(seed: int = SEED_BASE + 3, n_points: int = 512):
    """Per-point sizes of the mixed batch: M in {2,5,9,21}, K in {3,4}, N_t in {256,512,1024},
    N = floor(2^U(14,20))."""
    rng = np.random.default_rng(seed)
    M = rng.choice([2, 5, 9, 21], n_points)
    K = rng.choice([3, 4], n_points)
    Nt = rng.choice([256, 512, 1024], n_points)
    N = np.floor(2.0 ** rng.uniform(14, 20, n_points)).astype(np.int64)
    return [dict(n_det=int(K[i]), n_modes=int(M[i]), n_window=int(Nt[i]), n_samples=int(N[i]),
                 seed=seed * 1000 + i) for i in range(n_points)]
