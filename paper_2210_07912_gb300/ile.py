"""Thin ctypes binding of libile (include/ile.h).  Argument marshalling only: every step of the
hot path runs in the library's CUDA kernels.  There is no CPU fallback -- if libile.so is missing
or no CUDA device is present, every call raises.

Device arrays are passed as torch CUDA tensors (device memory and streams are the only things
PyTorch provides here); host arrays as numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ILE_OK, ILE_E_ARG, ILE_E_STATE, ILE_E_RANGE, ILE_E_NONFINITE, ILE_E_CUDA, ILE_E_NOMEM, ILE_E_TIMEOUT = range(8)
PREC = {"fp32": 0, "tf32x3": 1, "bf16x3": 2}
ILE_DEVICE_PTRS = 1
ILE_NO_TMARG = 2
ILE_NEAREST = 4
NDIM = 7
NBINS = 100
GMM_MAX = 8

_lib = None
ADAPT_LOG = 64


class AdaptCfg(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("point_id", ctypes.c_uint32), ("n_per_iter", ctypes.c_int64),
                ("n_iter", ctypes.c_int), ("adapt_mask", ctypes.c_uint), ("eps", ctypes.c_double),
                ("lo", ctypes.c_double * NDIM), ("hi", ctypes.c_double * NDIM), ("sky_frame", ctypes.c_int),
                ("sky_pole", ctypes.c_double * 3), ("gmm_mask", ctypes.c_uint), ("gmm_components", ctypes.c_int),
                ("gmm_em_iters", ctypes.c_int), ("gmm_pair", ctypes.c_int)]


class AdaptResult(ctypes.Structure):
    _fields_ = [("ln_L", ctypes.c_double), ("sigma_ln", ctypes.c_double), ("n_eff", ctypes.c_double),
                ("ess", ctypes.c_double), ("max_lnw", ctypes.c_double), ("s1", ctypes.c_double),
                ("s2", ctypes.c_double), ("n_total", ctypes.c_double), ("n_iter", ctypes.c_int),
                ("iter_ln_L", ctypes.c_double * ADAPT_LOG), ("iter_n_eff", ctypes.c_double * ADAPT_LOG),
                ("cdf", (ctypes.c_uint64 * (NBINS + 1)) * NDIM), ("hist", (ctypes.c_double * NBINS) * NDIM),
                ("gmm_components", ctypes.c_int * NDIM), ("gmm_w", (ctypes.c_double * GMM_MAX) * NDIM),
                ("gmm_mu", (ctypes.c_double * GMM_MAX) * NDIM), ("gmm_sigma", (ctypes.c_double * GMM_MAX) * NDIM),
                ("gmm_n", ctypes.c_double * NDIM), ("gmm_pair_components", ctypes.c_int),
                ("gmm_pair_w", ctypes.c_double * GMM_MAX), ("gmm_pair_mu", (ctypes.c_double * 2) * GMM_MAX),
                ("gmm_pair_cov", (ctypes.c_double * 3) * GMM_MAX), ("gmm_pair_n", ctypes.c_double)]


class PointDesc(ctypes.Structure):
    _fields_ = [("n_det", ctypes.c_int), ("n_modes", ctypes.c_int), ("lm", ctypes.c_void_p),
                ("det_tensor", ctypes.c_void_p), ("det_pos_m", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("T_ext", ctypes.c_int), ("t_start_s", ctypes.c_double), ("fs_hz", ctypes.c_double),
                ("U", ctypes.c_void_p), ("V", ctypes.c_void_p), ("n_window", ctypes.c_int),
                ("gmst_rad", ctypes.c_double), ("d_ref_mpc", ctypes.c_double), ("n_samples", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("point_id", ctypes.c_uint32), ("adapt_mask", ctypes.c_uint32),
                ("eps", ctypes.c_double), ("lo", ctypes.c_double * NDIM), ("hi", ctypes.c_double * NDIM),
                ("sky_frame", ctypes.c_int), ("sky_pole", ctypes.c_double * 3)]


TUNE_MAX = 32


class BatchTuning(ctypes.Structure):
    _fields_ = [("a_tmem", ctypes.c_int), ("nb", ctypes.c_int), ("nwcol", ctypes.c_int), ("grid", ctypes.c_int),
                ("ms", ctypes.c_float), ("n_tried", ctypes.c_int), ("tried_a_tmem", ctypes.c_int * TUNE_MAX),
                ("tried_nb", ctypes.c_int * TUNE_MAX), ("tried_nwcol", ctypes.c_int * TUNE_MAX),
                ("tried_ms", ctypes.c_float * TUNE_MAX)]


def default_ranges(fs: float = 4096.0, tc_max: float | None = None, d_min: float = 100.0, d_max: float = 1000.0):
    """Sampling-variable ranges (ra, sin dec, psi, cos iota, phi, D, t_c) of the extrinsic prior."""
    import math
    if tc_max is None:
        tc_max = 4.0 / fs
    return ([0.0, -1.0, 0.0, -1.0, 0.0, d_min, -tc_max], [2 * math.pi, 1.0, math.pi, 1.0, 2 * math.pi, d_max, tc_max])


def make_adapt_cfg(seed: int, n_per_iter: int, n_iter: int = 1, adapt_mask: int = 0b11, eps: float = 0.1,
                   point_id: int = 0, lo=None, hi=None, sky_pole=None, gmm_mask: int = 0, gmm_components: int = 3,
                   gmm_em_iters: int = 8, gmm_pair: bool = False) -> AdaptCfg:
    """sky_pole: Earth-fixed pole vector of the rotated network sky frame (e.g. r_L1 - r_H1); then
    sampling variables 0, 1 are (phi', sin lat') in that frame.  None: (ra, sin dec).
    gmm_mask: adaptive dimensions drawn from a truncated Gaussian mixture of gmm_components
    components, refit with gmm_em_iters EM steps per iteration.
    gmm_pair: sampling variables 0 and 1 drawn together from one correlated (bivariate) mixture."""
    dlo, dhi = default_ranges()
    lo = dlo if lo is None else lo
    hi = dhi if hi is None else hi
    pole = (0.0, 0.0, 0.0) if sky_pole is None else tuple(float(x) for x in sky_pole)
    return AdaptCfg(seed, point_id, n_per_iter, n_iter, adapt_mask, eps, (ctypes.c_double * NDIM)(*lo),
                    (ctypes.c_double * NDIM)(*hi), 0 if sky_pole is None else 1, (ctypes.c_double * 3)(*pole),
                    gmm_mask, gmm_components if (gmm_mask or gmm_pair) else 0,
                    gmm_em_iters if (gmm_mask or gmm_pair) else 0, 1 if gmm_pair else 0)


def result_dict(r: AdaptResult) -> dict:
    return dict(ln_L=r.ln_L, sigma_ln=r.sigma_ln, n_eff=r.n_eff, ess=r.ess, max_lnw=r.max_lnw, s1=r.s1, s2=r.s2,
                n_total=r.n_total, n_iter=r.n_iter, iter_ln_L=np.array(r.iter_ln_L[:max(r.n_iter, 0)]),
                iter_n_eff=np.array(r.iter_n_eff[:max(r.n_iter, 0)]),
                cdf=np.ctypeslib.as_array(r.cdf).copy(), hist=np.ctypeslib.as_array(r.hist).copy(),
                gmm=[None if r.gmm_components[d] == 0 else
                     dict(w=np.array(r.gmm_w[d][:r.gmm_components[d]]), mu=np.array(r.gmm_mu[d][:r.gmm_components[d]]),
                          sigma=np.array(r.gmm_sigma[d][:r.gmm_components[d]]), n=r.gmm_n[d])
                     for d in range(NDIM)],
                pair=None if r.gmm_pair_components == 0 else
                dict(w=np.array(r.gmm_pair_w[:r.gmm_pair_components]),
                     mu=np.array([[r.gmm_pair_mu[c][0], r.gmm_pair_mu[c][1]] for c in range(r.gmm_pair_components)]),
                     cov=np.array([[r.gmm_pair_cov[c][j] for j in range(3)] for c in range(r.gmm_pair_components)]),
                     n=r.gmm_pair_n))


class IleError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {_lib.ile_status_string(status).decode() if _lib else status}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libile.so (building it first if it is absent and nvcc exists).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libile.so not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i32, i64, d, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint
    P = ctypes.POINTER
    lib.ile_status_string.restype = ctypes.c_char_p
    lib.ile_status_string.argtypes = [i32]
    lib.ile_last_error.restype = ctypes.c_char_p
    lib.ile_last_error.argtypes = [vp]
    lib.ile_create.argtypes = [P(vp), i32, vp, i32]
    lib.ile_destroy.argtypes = [vp]
    lib.ile_set_stream.argtypes = [vp, vp]
    lib.ile_set_precision.argtypes = [vp, i32]
    lib.ile_set_data.argtypes = [vp, i32, i32, vp, vp, vp, vp, i32, d, d, vp, vp, i32, d, d]
    lib.ile_eval.argtypes = [vp, vp, i64, vp, u]
    lib.ile_integrate.argtypes = [vp, vp, vp, vp, i64, vp, vp, u]
    lib.ile_sync.argtypes = [vp]
    lib.ile_profile.argtypes = [vp, i32]
    lib.ile_profile_read.argtypes = [vp, vp, vp, i32]
    lib.ile_adapt_init.argtypes = [vp, P(AdaptCfg), P(AdaptResult)]
    lib.ile_adapt_step.argtypes = [vp, i32]
    lib.ile_adapt_get.argtypes = [vp, P(AdaptResult)]
    lib.ile_adapt_run.argtypes = [vp, P(AdaptCfg), P(AdaptResult)]
    lib.ile_adapt_last.argtypes = [vp, vp, vp, vp, vp]
    lib.ile_merge_partials.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp]
    lib.ile_merge_partials.restype = i32
    lib.ile_mc_reduce_noalloc.argtypes = [vp, vp, vp, i64, vp, vp]
    lib.ile_mc_reduce_noalloc.restype = i32
    lib.ile_set_refine.argtypes = [vp, i32]
    lib.ile_set_refine.restype = i32
    lib.ile_refine_count.argtypes = [vp, P(i64)]
    lib.ile_refine_count.restype = i32
    lib.ile_philox4x32_10.argtypes = [vp, i64, vp, vp]
    lib.ile_philox4x32_10.restype = i32
    lib.ile_batch_create.argtypes = [P(vp), i32, vp, i32]
    lib.ile_batch_destroy.argtypes = [vp]
    lib.ile_batch_set_points.argtypes = [vp, i32, P(PointDesc)]
    lib.ile_batch_reset.argtypes = [vp]
    lib.ile_batch_step.argtypes = [vp, i32]
    lib.ile_batch_get.argtypes = [vp, i32, i32, P(AdaptResult)]
    lib.ile_batch_run.argtypes = [vp, i32, P(PointDesc), i32, P(AdaptResult)]
    lib.ile_batch_last_samples.argtypes = [vp, i32, vp, vp]
    lib.ile_batch_config.argtypes = [vp, i32, i32, i32, i32]
    lib.ile_batch_tune.argtypes = [vp, i32, P(BatchTuning)]
    lib.ile_batch_last_error.argtypes = [vp]
    lib.ile_batch_last_error.restype = ctypes.c_char_p
    for name in ("ile_batch_create", "ile_batch_destroy", "ile_batch_set_points", "ile_batch_reset", "ile_batch_step",
                 "ile_batch_get", "ile_batch_run", "ile_batch_last_samples", "ile_batch_config", "ile_batch_tune"):
        getattr(lib, name).restype = i32
    lib.ile_set_distance_marginalization.argtypes = [vp, i32, d, d]
    lib.ile_set_distance_marginalization.restype = i32
    lib.ile_dmarg_eval.argtypes = [vp, vp, vp, i64, vp, u]
    lib.ile_build_quv.argtypes = [vp, i32, i32, i64, vp, vp, vp, d, d, d, d, i32, vp, vp, vp, u]
    lib.ile_build_quv.restype = i32
    lib.ile_dmarg_eval.restype = i32
    lib.ile_eval_grad.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, u]
    lib.ile_eval_grad.restype = i32
    lib.ile_integrate_grad.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, u]
    lib.ile_integrate_grad.restype = i32
    lib.ile_set_memory_limit.argtypes = [vp, ctypes.c_size_t]
    lib.ile_set_memory_limit.restype = i32
    lib.ile_memory_used.argtypes = [vp, P(ctypes.c_size_t)]
    lib.ile_memory_used.restype = i32
    lib.ile_check_wait_timeout.argtypes = [vp, d]
    lib.ile_check_wait_timeout.restype = i32
    for name in ("ile_create", "ile_destroy", "ile_set_stream", "ile_set_precision", "ile_set_data", "ile_eval",
                 "ile_integrate", "ile_sync", "ile_profile", "ile_profile_read", "ile_adapt_init", "ile_adapt_step",
                 "ile_adapt_get", "ile_adapt_run", "ile_adapt_last"):
        getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t):
    if t is None:
        return None
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("device tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


NOALLOC_MAX_SAMPLES = 1 << 22
GRAD_MAX_SAMPLES = 1 << 22


def merge_partials(max_lnw, s1, s2, n, hist=None):
    """Merge per-shard MC partial sums (host arrays, no GPU): dict like Context.integrate, plus the
    merged histograms if per-shard histograms ([shards][7][100]) are given."""
    lib = load()
    arrs = [np.ascontiguousarray(x, np.float64).reshape(-1) for x in (max_lnw, s1, s2, n)]
    k = arrs[0].size
    h = None if hist is None else np.ascontiguousarray(hist, np.float64).reshape(k, NDIM, NBINS)
    res = np.zeros(7)
    hout = None if h is None else np.zeros((NDIM, NBINS))
    st = lib.ile_merge_partials(k, *[_np_ptr(a) for a in arrs], _np_ptr(h), _np_ptr(res), _np_ptr(hout))
    if st != ILE_OK:
        raise IleError(st, "ile_merge_partials")
    d = dict(ln_L=res[0], sigma_ln=res[1], n_eff=res[2], ess=res[3], m=res[4], s1=res[5], s2=res[6])
    if hout is not None:
        d["hist"] = hout
    return d


def mc_reduce_noalloc(lnL_t, result, ln_prior=None, ln_ps=None, stream=None):
    """Monte Carlo reduction of per-sample device values into result[7] without any device
    allocation (for callers that cannot allocate; see include/ile.h).  All tensors are CUDA
    float64 on the current device; N = lnL_t.numel() must not exceed NOALLOC_MAX_SAMPLES.
    Queued on `stream` (torch stream or raw handle; None = legacy default stream)."""
    lib = load()
    import torch
    N = lnL_t.numel()
    if N > NOALLOC_MAX_SAMPLES:
        raise IleError(ILE_E_ARG, "ile_mc_reduce_noalloc",
                       f"N = {N} exceeds the fixed scratch of {NOALLOC_MAX_SAMPLES} samples")
    # the kernels read N doubles of every input and write 7 of result on the current device: refuse
    # anything else before it reaches them
    cur = torch.cuda.current_device()
    for name, t, need in (("lnL_t", lnL_t, N), ("ln_prior", ln_prior, N), ("ln_ps", ln_ps, N), ("result", result, 7)):
        if t is None:
            if name in ("lnL_t", "result"):
                raise IleError(ILE_E_ARG, "ile_mc_reduce_noalloc", f"{name} is required")
            continue
        if not t.is_cuda or t.device.index != cur or t.dtype != torch.float64 or not t.is_contiguous() \
                or t.numel() < need:
            raise IleError(ILE_E_ARG, "ile_mc_reduce_noalloc",
                           f"{name} must be a contiguous float64 CUDA tensor on device {cur} with >= {need} elements")
    st = lib.ile_mc_reduce_noalloc(_dev_ptr(lnL_t), _dev_ptr(ln_prior), _dev_ptr(ln_ps), N, _dev_ptr(result),
                                   _stream_handle(stream))
    if st != ILE_OK:
        raise IleError(st, "ile_mc_reduce_noalloc")


def philox4x32_10(ctr_key, out, stream=None):
    """Philox4x32-10 words of the device sampler's generator: ctr_key is a CUDA int32/uint32
    tensor [n][6] (counter words 0..3, key words 0..1), out a CUDA tensor [n][4] of the same
    dtype.  Queued on `stream` (None = legacy default stream)."""
    lib = load()
    n = ctr_key.shape[0]
    if ctr_key.shape != (n, 6) or out.shape != (n, 4) or not (ctr_key.is_cuda and out.is_cuda) \
            or ctr_key.element_size() != 4 or out.element_size() != 4:
        raise IleError(ILE_E_ARG, "ile_philox4x32_10", "ctr_key [n][6] and out [n][4] 32-bit CUDA tensors")
    st = lib.ile_philox4x32_10(_dev_ptr(ctr_key.contiguous()), n, _dev_ptr(out), _stream_handle(stream))
    if st != ILE_OK:
        raise IleError(st, "ile_philox4x32_10")


class Context:
    """One libile context (owns the device copy of one intrinsic point and its scratch)."""

    def __init__(self, device: int = 0, stream=None, prec: str = "fp32"):
        self._lib = load()
        self._h = ctypes.c_void_p()
        self._check(self._lib.ile_create(ctypes.byref(self._h), device, _stream_handle(stream), PREC[prec]),
                    "ile_create")
        self.device = device
        self.prec = prec
        self.n_window = None
        self.shape = (0, 0, 0)  # (K, M, T_ext) of the loaded point

    def _check(self, st, where):
        if st != ILE_OK:
            detail = self._lib.ile_last_error(self._h).decode() if self._h else ""
            raise IleError(st, where, detail)

    def close(self):
        if self._h:
            self._lib.ile_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_memory_limit(self, nbytes: int):
        """Cap the device memory this context may hold (0: no cap); past it calls raise ILE_E_NOMEM."""
        self._check(self._lib.ile_set_memory_limit(self._h, int(nbytes)), "ile_set_memory_limit")

    def memory_used(self) -> int:
        v = ctypes.c_size_t(0)
        self._check(self._lib.ile_memory_used(self._h, ctypes.byref(v)), "ile_memory_used")
        return v.value

    def check_wait_timeout(self, timeout_s: float = 0.05):
        """Run the bounded-wait check; raises IleError with ILE_E_TIMEOUT when the wait gives up."""
        self._check(self._lib.ile_check_wait_timeout(self._h, float(timeout_s)), "ile_check_wait_timeout")

    def set_stream(self, stream):
        self._check(self._lib.ile_set_stream(self._h, _stream_handle(stream)), "ile_set_stream")

    def set_refine(self, enable: bool = True):
        """FP64 refinement of loud samples (on by default; see ile_set_refine in include/ile.h)."""
        self._check(self._lib.ile_set_refine(self._h, 1 if enable else 0), "ile_set_refine")

    def refine_count(self) -> int:
        """Samples the last evaluation refined in FP64."""
        n = ctypes.c_int64()
        self._check(self._lib.ile_refine_count(self._h, ctypes.byref(n)), "ile_refine_count")
        return int(n.value)

    def set_precision(self, prec: str):
        self._check(self._lib.ile_set_precision(self._h, PREC[prec]), "ile_set_precision")
        self.prec = prec

    def set_data(self, p):
        lm = np.ascontiguousarray(p.lm, np.int32)
        tens = np.ascontiguousarray(p.det_tensor, np.float64)
        pos = np.ascontiguousarray(p.det_pos, np.float64)
        # complex128 arrays already hold (re, im) pairs in the [..][2] layout the library takes
        Q, U, V = (np.ascontiguousarray(x, np.complex128).view(np.float64) for x in (p.Q, p.U, p.V))
        K, M, T = p.Q.shape
        st = self._lib.ile_set_data(self._h, K, M, _np_ptr(lm), _np_ptr(tens), _np_ptr(pos), _np_ptr(Q), T,
                                    float(p.t_start), float(p.fs), _np_ptr(U), _np_ptr(V), int(p.n_window),
                                    float(p.gmst), float(p.d_ref))
        self._check(st, "ile_set_data")
        self.n_window = int(p.n_window)
        self.shape = (K, M, T)

    def set_distance_marginalization(self, enable: bool = True, d_min: float = 100.0, d_max: float = 1000.0):
        """Marginalise every returned likelihood over D (prior prop. to D^2 on [d_min, d_max])."""
        self._check(self._lib.ile_set_distance_marginalization(self._h, 1 if enable else 0, float(d_min),
                                                                float(d_max)), "ile_set_distance_marginalization")

    def build_quv(self, h, psd, d, df: float, f_low: float, t_start: float, fs: float, T_ext: int):
        """Q (K, M, T_ext), U, V (K, M, M) complex of Eq. (eq:QUV) from modes h (M, L), PSDs (K, L)
        and data d (K, L), two-sided frequency series in FFT order (host arrays)."""
        h = np.ascontiguousarray(np.stack([np.real(h), np.imag(h)], -1), np.float64)
        dd = np.ascontiguousarray(np.stack([np.real(d), np.imag(d)], -1), np.float64)
        S = np.ascontiguousarray(psd, np.float64)
        M, L = h.shape[:2]
        K = dd.shape[0]
        Q = np.zeros((K, M, T_ext, 2))
        U = np.zeros((K, M, M, 2))
        V = np.zeros((K, M, M, 2))
        self._check(self._lib.ile_build_quv(self._h, K, M, L, _np_ptr(h), _np_ptr(S), _np_ptr(dd), float(df),
                                            float(f_low), float(t_start), float(fs), int(T_ext), _np_ptr(Q),
                                            _np_ptr(U), _np_ptr(V), 0), "ile_build_quv")
        c = lambda x: x[..., 0] + 1j * x[..., 1]
        return c(Q), c(U), c(V)

    def dmarg_eval(self, a, b):
        """ln F(a, b) of the distance-marginalisation tables (host arrays)."""
        a = np.ascontiguousarray(a, np.float64)
        b = np.ascontiguousarray(np.broadcast_to(b, a.shape), np.float64)
        out = np.zeros_like(a)
        self._check(self._lib.ile_dmarg_eval(self._h, _np_ptr(a), _np_ptr(b), a.size, _np_ptr(out), 0),
                    "ile_dmarg_eval")
        return out

    # ---------------------------------------------------------------- host-pointer calls
    def eval(self, samples: np.ndarray, grid: bool = False, nearest: bool = False) -> np.ndarray:
        """lnL_t (or with grid=True the lnL(n, j) grid) of samples (7, N); nearest: Q at the nearest
        sample instead of the linear interpolation (ILE_NEAREST)."""
        s = np.ascontiguousarray(samples, np.float64)
        if s.ndim != 2 or s.shape[0] != NDIM:
            raise ValueError("samples must be (7, N)")
        N = s.shape[1]
        out = np.zeros((N, self.n_window) if grid else N, np.float64)
        flags = (ILE_NO_TMARG if grid else 0) | (ILE_NEAREST if nearest else 0)
        self._check(self._lib.ile_eval(self._h, _np_ptr(s), N, _np_ptr(out), flags), "ile_eval")
        return out

    def integrate(self, samples, ln_prior=None, ln_ps=None, want_lnL=False, nearest: bool = False):
        s = np.ascontiguousarray(samples, np.float64)
        N = s.shape[1]
        lp = None if ln_prior is None else np.ascontiguousarray(ln_prior, np.float64)
        lps = None if ln_ps is None else np.ascontiguousarray(ln_ps, np.float64)
        res = np.zeros(7)
        lnl = np.zeros(N) if want_lnL else None
        st = self._lib.ile_integrate(self._h, _np_ptr(s), _np_ptr(lp), _np_ptr(lps), N, _np_ptr(res), _np_ptr(lnl),
                                     ILE_NEAREST if nearest else 0)
        self._check(st, "ile_integrate")
        d = dict(ln_L=res[0], sigma_ln=res[1], n_eff=res[2], ess=res[3], m=res[4], s1=res[5], s2=res[6])
        return (d, lnl) if want_lnL else d

    # ---------------------------------------------------------------- device-pointer calls (async)
    def eval_device(self, samples, out, grid: bool = False):
        """samples: CUDA float64 (7, N); out: CUDA float64 (N,) or (N, N_t).  Queued on the context stream."""
        N = samples.shape[1]
        flags = ILE_DEVICE_PTRS | (ILE_NO_TMARG if grid else 0)
        self._check(self._lib.ile_eval(self._h, _dev_ptr(samples), N, _dev_ptr(out), flags), "ile_eval")

    def integrate_device(self, samples, result, ln_prior=None, ln_ps=None, lnL_out=None):
        N = samples.shape[1]
        st = self._lib.ile_integrate(self._h, _dev_ptr(samples), _dev_ptr(ln_prior), _dev_ptr(ln_ps), N,
                                     _dev_ptr(result), _dev_ptr(lnL_out), ILE_DEVICE_PTRS)
        self._check(st, "ile_integrate")

    def sync(self):
        self._check(self._lib.ile_sync(self._h), "ile_sync")

    # ---------------------------------------------------------------- gradients (adjoint kernels)
    def _grad_shapes(self):
        K, M, T = self.shape
        return (K, M, T, 2), (K, M, M, 2)

    def eval_grad(self, samples, g=None, want=("theta", "Q", "U", "V"), want_lnL=False):
        """Gradient of sum_n g[n] lnL_t(n) (host arrays): dict with the requested entries of
        theta (7, N), Q (K, M, T, 2), U and V (K, M, M, 2), and lnL (N,) if want_lnL."""
        s = np.ascontiguousarray(samples, np.float64)
        N = s.shape[1]
        gv = np.ones(N) if g is None else np.ascontiguousarray(g, np.float64)
        qs, us = self._grad_shapes()
        out = {}
        if "theta" in want:
            out["theta"] = np.zeros((NDIM, N))
        if "Q" in want:
            out["Q"] = np.zeros(qs)
        if "U" in want:
            out["U"] = np.zeros(us)
        if "V" in want:
            out["V"] = np.zeros(us)
        if want_lnL:
            out["lnL"] = np.zeros(N)
        st = self._lib.ile_eval_grad(self._h, _np_ptr(s), N, _np_ptr(gv), _np_ptr(out.get("theta")),
                                     _np_ptr(out.get("Q")), _np_ptr(out.get("U")), _np_ptr(out.get("V")),
                                     _np_ptr(out.get("lnL")), 0)
        self._check(st, "ile_eval_grad")
        return out

    def eval_grad_device(self, samples, g, g_theta=None, g_Q=None, g_U=None, g_V=None, lnL_out=None):
        """Device-pointer form of eval_grad (CUDA float64 tensors, queued on the context stream)."""
        N = samples.shape[1]
        st = self._lib.ile_eval_grad(self._h, _dev_ptr(samples), N, _dev_ptr(g), _dev_ptr(g_theta), _dev_ptr(g_Q),
                                     _dev_ptr(g_U), _dev_ptr(g_V), _dev_ptr(lnL_out), ILE_DEVICE_PTRS)
        self._check(st, "ile_eval_grad")

    def integrate_grad(self, samples, ln_prior=None, ln_ps=None, want=("theta", "Q", "U", "V")):
        """ln L_marg (dict as integrate) and its gradient through lnL_t (dict as eval_grad)."""
        s = np.ascontiguousarray(samples, np.float64)
        N = s.shape[1]
        lp = None if ln_prior is None else np.ascontiguousarray(ln_prior, np.float64)
        lps = None if ln_ps is None else np.ascontiguousarray(ln_ps, np.float64)
        qs, us = self._grad_shapes()
        out = {}
        if "theta" in want:
            out["theta"] = np.zeros((NDIM, N))
        if "Q" in want:
            out["Q"] = np.zeros(qs)
        if "U" in want:
            out["U"] = np.zeros(us)
        if "V" in want:
            out["V"] = np.zeros(us)
        res = np.zeros(7)
        st = self._lib.ile_integrate_grad(self._h, _np_ptr(s), _np_ptr(lp), _np_ptr(lps), N, None, _np_ptr(res),
                                          _np_ptr(out.get("theta")), _np_ptr(out.get("Q")), _np_ptr(out.get("U")),
                                          _np_ptr(out.get("V")), 0)
        self._check(st, "ile_integrate_grad")
        d = dict(ln_L=res[0], sigma_ln=res[1], n_eff=res[2], ess=res[3], m=res[4], s1=res[5], s2=res[6])
        return d, out

    def integrate_grad_device(self, samples, result, g_scale=None, ln_prior=None, ln_ps=None, g_theta=None,
                              g_Q=None, g_U=None, g_V=None):
        N = samples.shape[1]
        st = self._lib.ile_integrate_grad(self._h, _dev_ptr(samples), _dev_ptr(ln_prior), _dev_ptr(ln_ps), N,
                                          _dev_ptr(g_scale), _dev_ptr(result), _dev_ptr(g_theta), _dev_ptr(g_Q),
                                          _dev_ptr(g_U), _dev_ptr(g_V), ILE_DEVICE_PTRS)
        self._check(st, "ile_integrate_grad")

    # ---------------------------------------------------------------- adaptive integrator
    def adapt_init(self, cfg: AdaptCfg, resume: AdaptResult | None = None):
        self._check(self._lib.ile_adapt_init(self._h, ctypes.byref(cfg), ctypes.byref(resume) if resume else None),
                    "ile_adapt_init")
        self.adapt_N = cfg.n_per_iter

    def adapt_step(self, n_iter: int = 1):
        self._check(self._lib.ile_adapt_step(self._h, n_iter), "ile_adapt_step")

    def adapt_get(self, raw: bool = False):
        r = AdaptResult()
        self._check(self._lib.ile_adapt_get(self._h, ctypes.byref(r)), "ile_adapt_get")
        return r if raw else result_dict(r)

    def adapt_run(self, cfg: AdaptCfg, raw: bool = False):
        r = AdaptResult()
        self._check(self._lib.ile_adapt_run(self._h, ctypes.byref(cfg), ctypes.byref(r)), "ile_adapt_run")
        self.adapt_N = cfg.n_per_iter
        return r if raw else result_dict(r)

    def adapt_last(self):
        N = self.adapt_N
        theta = np.zeros((NDIM, N))
        lw = np.zeros(N)
        bins = np.zeros((NDIM, N), np.uint8)
        lnl = np.zeros(N)
        self._check(self._lib.ile_adapt_last(self._h, _np_ptr(theta), _np_ptr(lw), _np_ptr(bins), _np_ptr(lnl)),
                    "ile_adapt_last")
        return theta, lw, bins, lnl

    # ---------------------------------------------------------------- stage timing
    STAGES = ("sample", "prep", "contract", "mc", "adapt", "grad", "refine")

    def profile(self, enable: bool = True):
        self._check(self._lib.ile_profile(self._h, 1 if enable else 0), "ile_profile")

    def profile_read(self):
        """{stage: (total_ms, launches)} since the previous read (waits for the stream)."""
        ms = np.zeros(len(self.STAGES))
        cnt = np.zeros(len(self.STAGES), np.int64)
        self._check(self._lib.ile_profile_read(self._h, _np_ptr(ms), _np_ptr(cnt), len(self.STAGES)),
                    "ile_profile_read")
        return {s: (float(ms[i]), int(cnt[i])) for i, s in enumerate(self.STAGES)}


class Batch:
    """Batched adaptive run over many intrinsic points (ile_batch_*): one CUDA graph per
    iteration, the likelihood of all points in one persistent launch of the fused kernel."""

    def __init__(self, device: int = 0, stream=None, prec: str = "bf16x3"):
        self._lib = load()
        self._h = ctypes.c_void_p()
        self._check(self._lib.ile_batch_create(ctypes.byref(self._h), device, _stream_handle(stream), PREC[prec]),
                    "ile_batch_create")
        self.prec = prec
        self.n_points = 0
        self.sizes = []

    def _check(self, st, where):
        if st != ILE_OK:
            detail = self._lib.ile_batch_last_error(self._h).decode() if self._h else ""
            raise IleError(st, where, detail)

    def close(self):
        if self._h:
            self._lib.ile_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _descs(points, cfgs):
        keep, descs = [], (PointDesc * len(points))()
        for i, (p, c) in enumerate(zip(points, cfgs)):
            if c.gmm_mask:
                raise ValueError("batched runs adapt histograms only; Gaussian-mixture sampling is per point")
            lm = np.ascontiguousarray(p.lm, np.int32)
            tens = np.ascontiguousarray(p.det_tensor, np.float64)
            pos = np.ascontiguousarray(p.det_pos, np.float64)
            Q = np.ascontiguousarray(np.stack([p.Q.real, p.Q.imag], -1), np.float64)
            U = np.ascontiguousarray(np.stack([p.U.real, p.U.imag], -1), np.float64)
            V = np.ascontiguousarray(np.stack([p.V.real, p.V.imag], -1), np.float64)
            keep += [lm, tens, pos, Q, U, V]
            K, M, T = p.Q.shape
            d = descs[i]
            d.n_det, d.n_modes, d.T_ext, d.n_window = K, M, T, int(p.n_window)
            d.lm, d.det_tensor, d.det_pos_m = lm.ctypes.data, tens.ctypes.data, pos.ctypes.data
            d.Q, d.U, d.V = Q.ctypes.data, U.ctypes.data, V.ctypes.data
            d.t_start_s, d.fs_hz, d.gmst_rad, d.d_ref_mpc = float(p.t_start), float(p.fs), float(p.gmst), float(p.d_ref)
            d.n_samples, d.seed, d.point_id = c.n_per_iter, c.seed, c.point_id
            d.adapt_mask, d.eps = c.adapt_mask, c.eps
            for k in range(NDIM):
                d.lo[k], d.hi[k] = c.lo[k], c.hi[k]
            d.sky_frame = c.sky_frame
            for k in range(3):
                d.sky_pole[k] = c.sky_pole[k]
        return descs, keep

    def set_points(self, points, cfgs):
        """points: synthetic.Point list; cfgs: AdaptCfg per point (n_per_iter, seed, point_id, ...)."""
        descs, keep = self._descs(points, cfgs)
        self._check(self._lib.ile_batch_set_points(self._h, len(points), descs), "ile_batch_set_points")
        del keep
        self.n_points = len(points)
        self.sizes = [int(c.n_per_iter) for c in cfgs]

    def reset(self):
        self._check(self._lib.ile_batch_reset(self._h), "ile_batch_reset")

    def step(self, n_iter: int = 1):
        self._check(self._lib.ile_batch_step(self._h, n_iter), "ile_batch_step")

    def get(self, first: int = 0, count: int | None = None, raw: bool = False):
        count = self.n_points - first if count is None else count
        res = (AdaptResult * count)()
        self._check(self._lib.ile_batch_get(self._h, first, count, res), "ile_batch_get")
        return list(res) if raw else [result_dict(r) for r in res]

    def run(self, points, cfgs, n_iter: int, raw: bool = False):
        descs, keep = self._descs(points, cfgs)
        res = (AdaptResult * len(points))()
        self._check(self._lib.ile_batch_run(self._h, len(points), descs, n_iter, res), "ile_batch_run")
        del keep
        self.n_points = len(points)
        self.sizes = [int(c.n_per_iter) for c in cfgs]
        return list(res) if raw else [result_dict(r) for r in res]

    def last_samples(self, point: int):
        N = self.sizes[point]
        theta, lnl = np.zeros((NDIM, N)), np.zeros(N)
        self._check(self._lib.ile_batch_last_samples(self._h, point, _np_ptr(theta), _np_ptr(lnl)),
                    "ile_batch_last_samples")
        return theta, lnl

    def config(self, nb: int, nwcol: int, grid: int, a_tmem: int = 0):
        self._check(self._lib.ile_batch_config(self._h, a_tmem, nb, nwcol, grid), "ile_batch_config")

    def tune(self, reps: int = 3) -> dict:
        t = BatchTuning()
        self._check(self._lib.ile_batch_tune(self._h, reps, ctypes.byref(t)), "ile_batch_tune")
        tried = [(t.tried_a_tmem[i], t.tried_nb[i], t.tried_nwcol[i], float(t.tried_ms[i])) for i in range(t.n_tried)]
        return {"a_tmem": t.a_tmem, "nb": t.nb, "nwcol": t.nwcol, "grid": t.grid, "ms": float(t.ms), "tried": tried}
