/*
 * ile.h -- C ABI of libile, the GB300 (sm_103a) implementation of the ILE extrinsic-marginalisation
 * hot path of Wofford et al., "Expanding RIFT" (arXiv:2210.07912).
 *
 * For one intrinsic point (or a batch of points) and a set of Monte Carlo extrinsic samples
 * theta = (ra, dec, psi, iota, phi, D, t_c) the library computes
 *
 *   lnL(theta, j) = sum_k Re sum_lm conj(c_klm) Q_klm(t_k(j))
 *                   - 1/4 sum_k [ c_k^H U_k c_k + Re(c_k^T V_k c_k) ],     c_klm = (D_ref/D) F_k Y_lm
 *   lnL_t(theta)  = LSE_j lnL(theta, j) - ln N_t
 *   ln L_marg     = LSE_n [ lnL_t(theta_n) + ln p(theta_n) - ln p_s(theta_n) ] - ln N
 *
 * i.e. the likelihood decomposition of Eq. (eq:loglikelihood) with the inner products of
 * Eq. (eq:QUV) (App. "Numerical and adaptation approaches needed for strong signals"), the Monte
 * Carlo marginal likelihood of Eq. (eq:lnL:MonteCarlo) (Sec. "Evaluating the marginalized
 * likelihood"), summed in log space as in the subsection "Choices for finite-precision floating
 * point arithmetic and overflow", with the adaptive-Cartesian sampler of Sec. "GPU-accelerated
 * Monte Carlo integration" (separable sampling prior, 100-bin histograms per adaptive dimension).
 *
 * Conventions fixed here (the paper leaves them open):
 *   - F_k = F+ + i Fx from the detector response tensor D_k (3x3, Earth-fixed) in the textbook
 *     wave frame with X x Y = -n; Greenwich hour angle = gmst - ra.
 *   - Y_lm = _{-2}Y_lm(iota, phi) = sqrt((2l+1)/4pi) d^l_{m,2}(iota) e^{i m phi}.
 *   - t_k(j) = t_c + (j - N_t/2)/f_s + dt_k,  dt_k = -(r_k . n)/c; Q is sampled at
 *     t_start + i/f_s (i < T_ext) and linearly interpolated; every interpolation pair must lie
 *     inside [0, T_ext-1], otherwise the call returns ILE_E_RANGE.
 *   - The MC error is sigma_ln = sigma_I / I with the sample variance; n_eff = sum w / max w
 *     (Eq. (eq:neff)); ess = (sum w)^2 / sum w^2 (Eq. (eq:neff_ESS)).
 *
 * Ownership: the caller owns every buffer it passes.  ile_set_data copies its inputs into
 * context-owned device memory, so the caller may free them on return.  Outputs are written in
 * full, or not at all: a host-pointer call that fails (including a range, non-finite or timeout
 * error raised on the device) leaves the caller's output buffers untouched.
 *
 * Pointers: without ILE_DEVICE_PTRS every array argument is a host pointer and the call is
 * synchronous (it returns after the results are in host memory).  With ILE_DEVICE_PTRS they are
 * device pointers on the context's device, the work is queued on the context's stream and the
 * call returns at once; device-side errors (range, non-finite) are then reported by ile_sync().
 *
 * Errors: every call returns an ile_status and none aborts the process.  A CUDA error is mapped
 * to ILE_E_CUDA; the context stays usable if the CUDA context is intact.
 *
 * Threading: a context may be used by one host thread at a time.
 */
#ifndef ILE_H
#define ILE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ile_ctx ile_ctx; /* opaque; owns its device buffers */

typedef enum {
    ILE_OK = 0,
    ILE_E_ARG = 1,       /* invalid argument (null pointer, size out of range, bad mode list) */
    ILE_E_STATE = 2,     /* call out of order (e.g. ile_eval before ile_set_data) */
    ILE_E_RANGE = 3,     /* a sample's interpolation index left [0, T_ext-1] */
    ILE_E_NONFINITE = 4, /* a non-finite input sample or result */
    ILE_E_CUDA = 5,      /* CUDA runtime or launch error */
    ILE_E_NOMEM = 6,     /* device allocation failed */
    ILE_E_TIMEOUT = 7    /* a bounded device-side wait gave up */
} ile_status;

/* Arithmetic of the shifted contraction (S3); every other stage is the same in all modes.  Both
 * split precisions run the fused S1-S5 kernel (the quadratic term S4 as one more product per
 * detector in the same precision); TF32X3 keeps the coefficient operand in tensor memory and falls
 * back to an unfused kernel (S1, S2, S4 in FP32 on CUDA cores) for points with
 * n_det x (2 n_modes rounded up to 8) > 160. */
typedef enum {
    ILE_PREC_FP32 = 0,   /* FP32 CUDA-core GEMM ("plain") */
    ILE_PREC_TF32X3 = 1, /* tcgen05 kind::tf32, hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM */
    ILE_PREC_BF16X3 = 2  /* tcgen05 kind::f16 (bf16 operands), same three-product split */
} ile_prec;

/* flags */
#define ILE_DEVICE_PTRS 1u /* array arguments are device pointers; call is asynchronous */
#define ILE_NO_TMARG 2u    /* ile_eval writes lnL(n, j) for every window bin: out is [N][N_t] */
#define ILE_NEAREST 4u     /* ile_eval / ile_integrate: Q_k(t) at the nearest sample (ties to even)
                              instead of the linear interpolation between samples, for brute-force
                              cross-checks against a plain sum over the Q series */

#define ILE_NBINS 100      /* histogram bins per adaptive dimension (Sec. GPU-accelerated MC) */
#define ILE_NDIM 7         /* ra, dec, psi, iota, phi, D, t_c */
#define ILE_GMM_MAX 8      /* components per Gaussian-mixture dimension */
#define ILE_MAX_DET 4
#define ILE_MAX_MODES 21   /* all (l, m) with 2 <= l <= 4 */
#define ILE_MAX_WINDOW 1024
#define ILE_MAX_TEXT 4096

/* Create a context on CUDA device `device`.  cuda_stream is a cudaStream_t (NULL = legacy
 * default stream); the context never creates or destroys streams.  *out is NULL on failure. */
ile_status ile_create(ile_ctx **out, int device, void *cuda_stream, ile_prec prec);

/* Free every device buffer the context owns.  NULL is accepted. */
ile_status ile_destroy(ile_ctx *ctx);

/* Change the stream or the contraction arithmetic of an existing context. */
ile_status ile_set_stream(ile_ctx *ctx, void *cuda_stream);
ile_status ile_set_precision(ile_ctx *ctx, ile_prec prec);

/*
 * Load one intrinsic point (host pointers, copied).
 *   n_det in [1, 4]; n_modes in [1, 21]; lm: [n_modes][2] distinct (l, m), 2 <= l <= 4, |m| <= l.
 *   det_tensor: [n_det][3][3] response tensors; det_pos_m: [n_det][3] vertex positions (m).
 *   Q: [n_det][n_modes][T_ext][2] (re, im) = <h_lm(t_i) | d>_k at t_i = t_start_s + i / fs_hz.
 *   U, V: [n_det][n_modes][n_modes][2], U_k Hermitian, V_k symmetric (Eq. (eq:QUV)).
 *   n_window = N_t in [1, 1024]; T_ext in [2, 4096]; fs_hz > 0; d_ref_mpc > 0.
 * May be called again to replace the point.  Returns ILE_E_ARG or ILE_E_NONFINITE for a bad
 * argument; the previous point is kept after an ILE_E_ARG and after a non-finite detector
 * description, U or V, but a non-finite Q (checked on the device while it is converted) leaves
 * the context without data (ILE_E_STATE until the next successful call).
 */
ile_status ile_set_data(ile_ctx *ctx, int n_det, int n_modes, const int *lm, const double *det_tensor,
                        const double *det_pos_m, const double *Q, int T_ext, double t_start_s, double fs_hz,
                        const double *U, const double *V, int n_window, double gmst_rad, double d_ref_mpc);

/*
 * Refinement of loud samples (the subsection "Choices for finite-precision floating point
 * arithmetic and overflow" keeps the likelihood in log space so that loud signals, SNR rho ~ 35 and
 * beyond, do not overflow; this keeps them accurate too).  Every fast path computes geometry,
 * coefficients and the data and quadratic terms in single precision (or split precision on the
 * tensor cores), whose absolute error grows with |D| + A: measured against the FP64 oracle, below
 * 1e-6 (FP32, TF32X3) and 5e-6 (BF16X3) of |max_j D| + A.  With refinement on (the default), a
 * sample with |max_j D| + A above 300 (FP32, TF32X3) or 50 (BF16X3) is recomputed on the device:
 * geometry, harmonics, coefficients and A in FP64 from FP64 copies of the point, every window bin's
 * data term in FP32, and in FP64 every bin with D_j >= max_j D - 30 and |D_j| above the same
 * threshold; its lnL_t is then the FP64 log-sum-exp of those bins.  Applies to ile_eval (lnL_t),
 * ile_integrate, the adaptive integrator and the batched run, not to the lnL(n, j) grid, the
 * adjoint or the distance-marginalised likelihood.  Costs one small launch per evaluation when no
 * sample is loud; the FP64 work of a loud sample is a few ten thousand FP64 operations.
 *   ile_set_refine: enable (1, default) or disable (0) it for the context.
 *   ile_refine_count: waits for the context's stream; *n = the number of samples the last
 *   evaluation refined (the last iteration's, after ile_adapt_step).
 */
ile_status ile_set_refine(ile_ctx *ctx, int enable);
ile_status ile_refine_count(ile_ctx *ctx, int64_t *n);

/*
 * Distance marginalisation (App. "Distance marginalization"; the paper gives no formula, the
 * integral is written out here).  When enabled, every likelihood the context returns (ile_eval,
 * ile_integrate, the adaptive integrator) is marginalised over the luminosity distance:
 *   lnL_D(n) = ln (1/N_t) sum_j F(a_j, b) ,  F(a, b) = int p(D) exp(a x - b x^2) dD ,  x = D_ref / D,
 * p(D) = 3 D^2 / (D_max^3 - D_min^3) on [d_min_mpc, d_max_mpc], with a_j the data term of window
 * bin j and b the quadratic term, both at D = D_ref; the samples' own distance is ignored (the
 * Monte Carlo then integrates over the other six parameters; give D a fixed, non-adaptive range).
 * ln F comes from two tables (b < 10: ln F on an (a, b) grid; b >= 10: ln F minus its peak
 * exponent on a grid in the standardised peak position and ln b; about 28 MB of device memory,
 * built in FP64 on the device when this is called) with bilinear interpolation; the quadratic term
 * b is covered up to 10^6.  The adjoint entry points return ILE_E_STATE while it is enabled.
 * Requires ile_set_data; ile_set_data turns it off.  0 < d_min_mpc < d_max_mpc.
 */
ile_status ile_set_distance_marginalization(ile_ctx *ctx, int enable, double d_min_mpc, double d_max_mpc);

/*
 * The inner-product arrays of Eq. (eq:QUV) of one intrinsic point, in FP64 on the device, from
 * the mode waveforms, the detectors' noise PSDs and data (frequency domain, two-sided, L bins in
 * FFT order: bin m is f = m df for m < L/2, (m - L) df otherwise):
 *   Q[k][a][i] = 2 df sum_{|f|>f_low} e^{2 pi i f t_i} conj(h_a(f)) d_k(f) / S_k(f),
 *                t_i = t_start_s + i / fs_hz, i < T_ext;
 *   U[k][a][b] = 2 df sum_{|f|>f_low} conj(h_a(f)) h_b(f) / S_k(f);
 *   V[k][a][b] = 2 df sum_{|f|>f_low} h_a(-f) h_b(f) / S_k(f)   (<h_a^* | h_b>).
 *   h: [n_modes][L][2]; psd: [n_det][L] (S_k at |f| of each bin); d: [n_det][L][2];
 *   Q: [n_det][n_modes][T_ext][2], U, V: [n_det][n_modes][n_modes][2] -- the layouts
 *   ile_set_data takes.  flags: ILE_DEVICE_PTRS (else host arrays).  Synchronous; allocates
 *   16 K M L bytes of scratch for the call.  2 <= L <= 2^24; f_low < 0 keeps every bin.
 */
ile_status ile_build_quv(ile_ctx *ctx, int n_det, int n_modes, int64_t L, const double *h, const double *psd,
                         const double *d, double df, double f_low, double t_start_s, double fs_hz, int T_ext,
                         double *Q, double *U, double *V, unsigned flags);

/* ln F(a[i], b[i]) from the context's distance-marginalisation tables (the per-bin term of the
 * distance-marginalised likelihood), for inspection and tests.  ILE_E_STATE unless enabled.
 * flags: ILE_DEVICE_PTRS (else host arrays, synchronous). */
ile_status ile_dmarg_eval(ile_ctx *ctx, const double *a, const double *b, int64_t n, double *out, unsigned flags);

/*
 * Time-marginalised log-likelihood of N samples (S1-S5).
 *   samples: SoA [7][N] (ra, dec, psi, iota, phi, D_Mpc, tc_s), FP64.
 *   out: lnL_t [N] FP64, or with ILE_NO_TMARG lnL [N][N_t] FP64 (then N <= 65536).
 * N = 0 is a valid no-op.
 */
ile_status ile_eval(ile_ctx *ctx, const double *samples, int64_t N, double *out, unsigned flags);

/*
 * Monte Carlo marginal likelihood of Eq. (eq:lnL:MonteCarlo) over N samples (S1-S6).
 *   ln_prior, ln_ps: [N] log prior and log sampling densities of each sample (same coordinates).
 *   result (7 doubles): {ln L_marg, sigma_ln, n_eff, ess, max ln w, S1, S2} with
 *   S1 = sum exp(ln w - max), S2 = sum exp(2 (ln w - max)) (the mergeable partial sums).
 *   lnL_t_out (optional, may be NULL): the per-sample lnL_t [N].
 * Requires N >= 1.
 */
ile_status ile_integrate(ile_ctx *ctx, const double *samples, const double *ln_prior, const double *ln_ps,
                         int64_t N, double *result, double *lnL_t_out, unsigned flags);

/* ------------------------------------------------------------------ adaptive MC integrator */

/*
 * Adaptive-Cartesian integrator (Sec. "GPU-accelerated Monte Carlo integration"): every
 * iteration draws n_per_iter samples on the device from the separable sampling prior
 * p_s = prod_d p_{s,d}, evaluates lnL_t, accumulates the Monte Carlo sums of
 * Eq. (eq:lnL:MonteCarlo) (pooled over iterations, each sample weighted with the p_s it was drawn
 * from) and refits the 100-bin histogram of every adaptive dimension.
 *   Sampling variables d = 0..6: ra, sin(dec), psi, cos(iota), phi, D (Mpc), t_c (s), on
 *   [lo[d], hi[d]]; the prior is uniform in each, except D (prop. to D^2).  A fixed dimension is
 *   drawn from its prior; an adaptive one (bit d of adapt_mask) from its histogram.
 *   Random numbers: Philox4x32-10 with key = seed and counter (sample index, iteration, point_id,
 *   block), so a run (or a resumed run) is reproducible bit for bit.
 *   Histogram update: mass_b = (1 - eps) h_b / sum h + eps / 100, h_b the sum of the weights of
 *   the iteration's samples in bin b; eps in (0, 1].
 */
/*
 * Rotated detector-network-frame sky coordinates (Sec. on coordinate choices, "rotated
 * detector-network-frame sky coordinates"): with sky_frame = 1 the first two sampling variables
 * are the longitude phi' and sin(latitude') in a frame whose north pole is sky_pole (Earth-fixed,
 * typically the baseline between two detectors, along which lines of constant latitude are lines
 * of constant time delay).  Frame: p = pole / |pole|, e1 = z x p / |z x p| (x when p is along z),
 * e2 = p x e1; the source direction n = cos(lat') cos(phi') e1 + cos(lat') sin(phi') e2 +
 * sin(lat') p, then dec = asin(n_z), ra = gmst - atan2(-n_y, n_x) in [0, 2 pi).  The uniform sky
 * prior is the same density in either frame; the histograms adapt in the rotated variables.
 */
/*
 * Gaussian-mixture sampling (Sec. "Adaptive sampling with gaussian mixture models", App.
 * "Gaussian mixture model implementation"), separable form: an adaptive dimension d in gmm_mask
 * is drawn from p_{s,d}(u) = sum_c w_c N(u | mu_c, sigma_c) / Z_c, each normal truncated to
 * [lo_d, hi_d] (Z_c its mass there), instead of from a histogram.
 *   Sampling: the component is the largest c with cw[c] <= a (cw the integer cumulative weight
 *   table, 2^32 scale, built like the histogram tables), then u = mu_c + sigma_c Phi^-1(P1 + v
 *   (P2 - P1)), P1, P2 = Phi((lo - mu_c) / sigma_c), Phi((hi - mu_c) / sigma_c), v from the
 *   second word; bins[d] holds the component.
 *   Update, every iteration: gmm_em_iters EM steps on the iteration's samples, started from the
 *   current mixture, with responsibilities r_nc prop. to w_c N(u_n | mu_c, sigma_c) and sample
 *   weights w_n = exp(ln w_n - max): S0_c = sum_n w_n r_nc, mu_c = sum w r u / S0_c,
 *   sigma_c^2 = sum w r (u - mu_c)^2 / S0_c (at least (1e-3 (hi - lo))^2), w_c = S0_c / sum w_n
 *   (a component with S0_c <= 1e-12 sum w keeps mu, sigma and gets weight 1e-3; weights are
 *   renormalised).  Then the online merge: batch component i is paired with current component j
 *   by the permutation of least sum |mu_i - mu_j| (1 / sigma_i + 1 / sigma_j) (the first such
 *   permutation in lexicographic order), and each pair combined with N = samples the current
 *   mixture was trained on, M = n_per_iter: mu = (N w_j mu_j + M w_i mu_i) / (N w_j + M w_i),
 *   sigma^2 = (N w_j (sigma_j^2 + mu_j^2) + M w_i (sigma_i^2 + mu_i^2)) / (N w_j + M w_i) - mu^2,
 *   w = (N w_j + M w_i) / (N + M); then N <- N + M.
 *   Start: gmm_components equal components, means at the centres of equal slices of [lo, hi],
 *   sigma = (hi - lo) / C, N = 0 (so the first merge keeps the batch mixture); or the mixtures of
 *   a resumed ile_adapt_result.
 */
/*
 * Correlated sampling of the sky pair (the same section: correlated sampling in a chosen subset of
 * dimensions, with the multivariate EM, merge and rejection to the finite domain of App. "Gaussian
 * mixture model implementation"): with gmm_pair = 1, sampling variables 0 and 1 (ra and sin dec,
 * or the rotated frame's longitude and sin latitude) are drawn together from
 *   p_s(x) = sum_c w_c N(x | mu_c, S_c) / Z_c  on the rectangle R = [lo0, hi0] x [lo1, hi1],
 * each component a bivariate normal truncated to R, Z_c its mass in R (computed by quadrature of
 * the conditional normal, so ln p_s is exact and the integral unbiased).
 *   Sampling: the component is the largest c with cw[c] <= a (a = word 0 of the sample); then
 *   attempt t = 0, 1, ... takes Philox block 4 + t of the sample's counter, two standard normals
 *   y truncated to the box that holds L_c^-1 (R - mu_c) (L_c the Cholesky factor of S_c, inverse
 *   CDF from the nearer tail) and x = mu_c + L_c y; the first x inside R is kept (1024 attempts at
 *   most, else ILE_E_RANGE).  bins[0] = bins[1] = c.
 *   Update, every iteration: gmm_em_iters EM steps on the iteration's pairs with r_nc prop. to
 *   w_c N(x_n | mu_c, S_c) and weights w_n = exp(ln w_n - max): S0_c = sum w_n r_nc, mu_c, S_c
 *   the weighted mean and covariance, w_c = S0_c / sum w_n; then sigma_j >= 1e-3 (hi_j - lo_j),
 *   |rho| <= 0.9 and mu_c inside R.  The merge pairs batch and current components by the least
 *   sum of sqrt(d^T S_i^-1 d) + sqrt(d^T S_j^-1 d) (d = mu_j - mu_i; first least permutation) and
 *   combines them with N and M as for one dimension, S = (N w_j S_j + M w_i S_i) / (...) +
 *   (N w_j mu_j mu_j^T + M w_i mu_i mu_i^T) / (...) - mu mu^T, followed by the same limits.
 *   Start: C components with means on R's diagonal at the centres of C equal slices, standard
 *   deviations (hi_j - lo_j) / C, no correlation, N = 0; or gmm_pair_* of a resumed result.
 *   Requires bits 0 and 1 of adapt_mask and not of gmm_mask.
 */
typedef struct {
    uint64_t seed;
    uint32_t point_id;
    int64_t n_per_iter;   /* samples per iteration, 1 .. 2^23 */
    int n_iter;           /* iterations run by ile_adapt_run */
    unsigned adapt_mask;  /* bit d: dimension d adaptive */
    double eps;           /* histogram floor, (0, 1] */
    double lo[ILE_NDIM], hi[ILE_NDIM];
    int sky_frame;        /* 0: sky variables 0, 1 are (ra, sin dec); 1: rotated network frame */
    double sky_pole[3];   /* sky_frame 1: Earth-fixed vector of the frame's pole (e.g. r_L1 - r_H1) */
    unsigned gmm_mask;    /* bits of adapt_mask drawn from a Gaussian mixture; 0: histograms only */
    int gmm_components;   /* gmm_mask != 0 or gmm_pair: components per mixture, 1 .. ILE_GMM_MAX */
    int gmm_em_iters;     /* gmm_mask != 0 or gmm_pair: EM steps per iteration, 1 .. 100 */
    int gmm_pair;         /* 1: sampling variables 0 and 1 (the sky pair) from one correlated mixture */
} ile_adapt_cfg;

#define ILE_ADAPT_LOG 64
typedef struct {
    double ln_L, sigma_ln, n_eff, ess;   /* pooled estimate over every iteration so far */
    double max_lnw, s1, s2, n_total;     /* pooled partial sums: S1 = sum e^{ln w - max}, S2 = sum e^{2(...)} */
    int n_iter;                          /* iterations done (the Philox iteration counter) */
    double iter_ln_L[ILE_ADAPT_LOG];     /* per-iteration ln L estimate (first 64 iterations) */
    double iter_n_eff[ILE_ADAPT_LOG];    /* per-iteration n_eff */
    uint64_t cdf[ILE_NDIM][ILE_NBINS + 1]; /* current integer cumulative tables (2^32 scale) */
    double hist[ILE_NDIM][ILE_NBINS];    /* last iteration's weight histograms (relative to its max) */
    int gmm_components[ILE_NDIM];        /* mixture dimensions: components; 0 otherwise */
    double gmm_w[ILE_NDIM][ILE_GMM_MAX], gmm_mu[ILE_NDIM][ILE_GMM_MAX], gmm_sigma[ILE_NDIM][ILE_GMM_MAX];
    double gmm_n[ILE_NDIM];              /* samples each mixture has been trained on */
    int gmm_pair_components;             /* the sky pair's correlated mixture (gmm_pair): components */
    double gmm_pair_w[ILE_GMM_MAX], gmm_pair_mu[ILE_GMM_MAX][2];
    double gmm_pair_cov[ILE_GMM_MAX][3]; /* {S00, S01, S11} of each component */
    double gmm_pair_n;
} ile_adapt_result;

/* Set up the sampler on the current point (after ile_set_data).  resume = NULL starts from uniform
 * tables, the initial mixtures and empty sums; otherwise the tables, mixtures, sums and iteration
 * counter of `resume` are loaded (checkpoint/resume).  ILE_E_ARG for a bad configuration:
 * gmm_mask not inside adapt_mask, components or EM steps out of range, or a resumed mixture with
 * another component count, a weight <= 0, a sigma <= 0 or a mean outside [lo, hi]. */
ile_status ile_adapt_init(ile_ctx *ctx, const ile_adapt_cfg *cfg, const ile_adapt_result *resume);
/* Queue n_iter iterations on the context stream (asynchronous). */
ile_status ile_adapt_step(ile_ctx *ctx, int n_iter);
/* Wait for the stream and read the integrator state. */
ile_status ile_adapt_get(ile_ctx *ctx, ile_adapt_result *out);
/* ile_adapt_init(cfg, NULL) + ile_adapt_step(cfg->n_iter) + ile_adapt_get. */
ile_status ile_adapt_run(ile_ctx *ctx, const ile_adapt_cfg *cfg, ile_adapt_result *out);
/* Copy the last iteration's samples to host memory (any pointer may be NULL):
 * theta [7][N], ln p - ln p_s [N], bins [7][N] (255 for fixed dimensions), lnL_t [N]. */
ile_status ile_adapt_last(ile_ctx *ctx, double *theta, double *lnw_prior, uint8_t *bins, double *lnL_t);

/*
 * Stage timing (tracing aid): when enabled, every kernel launch of the context is bracketed by
 * CUDA events recorded on the context's stream.  ile_profile_read waits for the stream and
 * writes, for each stage s < n_stages, the summed device time in ms (out_ms[s]) and the number
 * of kernel launches (out_count[s], may be NULL) since the previous read, then resets them.
 * Stages: 0 sampler (S0), 1 geometry/coefficients/quadratic (S1, S2, S4), 2 shifted contraction
 * and time log-sum-exp (S3, S5), 3 Monte Carlo reduction (S6), 4 histogram adaptation (S6),
 * 5 adjoint (ile_eval_grad / ile_integrate_grad), 6 FP64 refinement of loud samples.
 */
#define ILE_NSTAGE 7
ile_status ile_profile(ile_ctx *ctx, int enable);
ile_status ile_profile_read(ile_ctx *ctx, double *out_ms, int64_t *out_count, int n_stages);

/*
 * Allocation-free Monte Carlo reduction (the paper has no counterpart; this is a service for
 * callers that cannot allocate device memory, e.g. code running inside another framework's
 * memory pool, a CUDA-graph capture region or a pre-sized real-time service, where a cudaMalloc
 * would synchronise the device or is not permitted).
 *
 * Computes the same result[7] as ile_integrate (ln L_marg, sigma_ln, n_eff, ess, max ln w, S1,
 * S2) from per-sample values that are already on the device: ln w_n = lnL_t[n] + ln_prior[n] -
 * ln_ps[n] (ln_prior / ln_ps may be NULL, meaning 0).  All pointers are device pointers on the
 * current CUDA device; the work is queued on cuda_stream (a cudaStream_t; NULL = legacy default
 * stream) and the call returns without waiting.  It needs no context and allocates nothing: its
 * scratch (the per-block partial sums) is a fixed array inside the library, 24 KB on every
 * device that loads the library, kept as long as the CUDA context that loaded it (normally until
 * the process exits).
 *   N must be in [1, ILE_NOALLOC_MAX_SAMPLES]; larger N returns ILE_E_ARG (use ile_integrate).
 *   Every call looks up the array's device address (cudaGetSymbolAddress), so the entry point
 *   keeps working after cudaDeviceReset; the first call on a device may load the library's device
 *   code into the context, so make that first call before capturing a stream into a CUDA graph.
 *   Every call shares the one array: calls whose work overlaps on the GPU (on different streams,
 *   or from different host threads without ordering) race and may return wrong results.
 *   Returns ILE_E_CUDA if the device address cannot be obtained or a launch fails.
 */
#define ILE_NOALLOC_MAX_SAMPLES (1 << 22)
ile_status ile_mc_reduce_noalloc(const double *lnL_t, const double *ln_prior, const double *ln_ps, int64_t N,
                                 double *result, void *cuda_stream);

/*
 * Merge per-shard Monte Carlo partial sums (host memory, no GPU needed).  The path shards over
 * samples and over intrinsic points with one exchange: each shard s reports (max_s, S1_s, S2_s,
 * n_s) with S1 = sum e^{ln w - max}, S2 = sum e^{2(ln w - max)} (result[4..6] of ile_integrate and
 * the pooled fields of ile_adapt_result) and optionally its weight histograms hist_s[7][100]
 * (relative to the same max).  Writes result[7] = {ln L_marg, sigma_ln, n_eff, ess, max, S1, S2}
 * of the union of the shards, and (if hist_out is not NULL) the merged histograms relative to the
 * merged max.  Shards with n_s = 0 are ignored; ILE_E_ARG if no shard has samples.
 */
ile_status ile_merge_partials(int n_shards, const double *max_lnw, const double *s1, const double *s2,
                              const double *n, const double *hist /* [n_shards][7][100] or NULL */,
                              double *result, double *hist_out /* [7][100] or NULL */);

/* ------------------------------------------------------------------ batched adaptive run */

#define ILE_BATCH_MAX_POINTS 4096
#define ILE_TUNE_MAX 32

/* One intrinsic point of a batch: the ile_set_data arguments plus its sampler (as in
 * ile_adapt_cfg; n_iter is given to ile_batch_step instead).  Host pointers, copied by
 * ile_batch_set_points. */
typedef struct {
    int n_det, n_modes;
    const int *lm;
    const double *det_tensor, *det_pos_m, *Q;
    int T_ext;
    double t_start_s, fs_hz;
    const double *U, *V;
    int n_window;
    double gmst_rad, d_ref_mpc;
    int64_t n_samples; /* samples per iteration, 1 .. 2^23 */
    uint64_t seed;
    uint32_t point_id;
    uint32_t adapt_mask;
    double eps;
    double lo[ILE_NDIM], hi[ILE_NDIM];
    int sky_frame;
    double sky_pole[3];
} ile_point_desc;

typedef struct ile_batch ile_batch; /* opaque; owns the device copies of all points */

/* Result of ile_batch_tune: the chosen configuration of the fused kernel (placement of the MMA A
 * operand a_tmem: 0 shared memory, 1 tensor memory; B-ring depth nb; job window width nwcol in
 * time columns; persistent CTAs grid), its time per launch, and every combination tried. */
typedef struct {
    int a_tmem, nb, nwcol, grid;
    float ms;
    int n_tried;
    int tried_a_tmem[ILE_TUNE_MAX], tried_nb[ILE_TUNE_MAX], tried_nwcol[ILE_TUNE_MAX];
    float tried_ms[ILE_TUNE_MAX];
} ile_batch_tuning;

/*
 * Batched adaptive Monte Carlo integration of many intrinsic points (each with its own Q/U/V,
 * detectors, modes, window, sample budget and sampler), Sec. "GPU-accelerated Monte Carlo
 * integration" applied point by point.  Per iteration, all points are sampled, delay-sorted,
 * evaluated and their integrals and histograms updated by a fixed launch sequence captured once
 * in a CUDA graph; with ILE_PREC_BF16X3 the likelihood of every (point, 128-sample tile) work item
 * runs in ONE persistent launch of the fused tensor-core kernel, longest items first.  Each
 * point's result equals (bit for bit) an ile_adapt_run of that point alone with the same seed,
 * point_id and ranges.
 *   ile_batch_create: cuda_stream NULL = a stream owned by the batch (graphs cannot be captured
 *     on the legacy default stream).
 *   ile_batch_set_points: copies and validates every point (ILE_E_ARG / ILE_E_NONFINITE as
 *     ile_set_data and ile_adapt_init), allocates the per-sample arrays (about 90 bytes per
 *     sample per iteration) and resets every sampler.  1 <= n_points <= ILE_BATCH_MAX_POINTS.
 *   ile_batch_reset: uniform tables, empty accumulators, iteration 0 for every point.
 *   ile_batch_step: queue n_iter iterations (asynchronous on the batch stream).
 *   ile_batch_get: results of points first .. first + count - 1 (waits for the stream; returns
 *     the first device-side error, as ile_sync).
 *   ile_batch_run: set_points + step(n_iter) + get of all points; out has n_points entries.
 *   ile_batch_last_samples: the last iteration's samples [7][N] and lnL_t [N] of one point (host).
 *   ile_batch_config: set the fused kernel's configuration by hand: a_tmem 0 keeps the MMA A
 *     operand (the tile's coefficients) in shared memory with three 128-column TMEM accumulator
 *     buffers (window widths 66 .. 121), a_tmem 1 puts it in tensor memory with two 160-column
 *     buffers (widths 66 .. 153; every point needs n_det x (2 n_modes rounded up to 16) <= 192),
 *     the B-ring depth (2..4, if it fits in shared memory), the window width and the CTA count;
 *     ILE_E_ARG otherwise.  Every configuration gives the same results bit for bit.
 *   ile_batch_tune: autotuner -- runs one iteration to have samples, then times the fused
 *     kernel over that iteration's work items (a timed warm-up launch per candidate, then reps
 *     timed launches unless the warm-up already took more than twice the best time; reps >= 3
 *     recommended): for each A placement that fits, every window width nwcol on an 8-column grid
 *     over its admissible range (both ends included, widest first) at the deepest B ring that
 *     fits, then each shallower ring at that placement's best width; keeps the fastest (BF16X3
 *     only; else ILE_E_STATE).  The grid stays one persistent CTA per SM (the kernel holds a
 *     whole SM).  The sampler advances by one iteration: call ile_batch_reset before the run that
 *     counts.
 */
ile_status ile_batch_create(ile_batch **out, int device, void *cuda_stream, ile_prec prec);
ile_status ile_batch_destroy(ile_batch *b);
ile_status ile_batch_set_points(ile_batch *b, int n_points, const ile_point_desc *points);
ile_status ile_batch_reset(ile_batch *b);
ile_status ile_batch_step(ile_batch *b, int n_iter);
ile_status ile_batch_get(ile_batch *b, int first, int count, ile_adapt_result *out);
ile_status ile_batch_run(ile_batch *b, int n_points, const ile_point_desc *points, int n_iter,
                         ile_adapt_result *out);
ile_status ile_batch_last_samples(ile_batch *b, int point, double *theta, double *lnL_t);
ile_status ile_batch_config(ile_batch *b, int a_tmem, int nb, int nwcol, int grid);
ile_status ile_batch_tune(ile_batch *b, int reps, ile_batch_tuning *out);
const char *ile_batch_last_error(const ile_batch *b);

/* ------------------------------------------------------------------ gradients (adjoint) */

#define ILE_GRAD_MAX_SAMPLES (1 << 22)

/*
 * Gradient of sum_n g_lnL[n] lnL_t(n) (the vector-Jacobian product of ile_eval) by hand-written
 * adjoint kernels.  The paper gives no derivative: this is the exact derivative of the
 * time-marginalised likelihood of Eq. (eq:loglikelihood) as computed (linear interpolation of Q
 * differentiated inside the bin the window start falls in), in FP32 per sample with FP64 sums
 * over samples; the coefficient stage is recomputed from the samples.  The context's precision
 * selects the contractions: FP32 contexts recompute the data term and contract on CUDA cores;
 * BF16x3 contexts take the data term from the fused tensor-core forward kernel and run the
 * E / interpolation-slope and dQ contractions as BF16x3 tensor-core GEMMs (FP32 accumulation).
 *   samples: SoA [7][N] FP64 as in ile_eval; g_lnL: [N] upstream weights.
 *   g_samples: [7][N] d/d(ra, dec, psi, iota, phi, D_Mpc, tc_s) of each sample, times g_lnL[n].
 *   g_Q: [n_det][n_modes][T_ext][2]; g_U, g_V: [n_det][n_modes][n_modes][2]: derivatives with
 *   respect to the real and imaginary part of every entry, the entries taken as independent
 *   (no Hermitian or symmetric tying), summed over the samples.  U and V themselves must be
 *   Hermitian / symmetric as ile_set_data requires.
 *   lnL_t_out: [N] lnL_t recomputed by the adjoint's forward pass.
 * Any output may be NULL (at least one is required); 1 <= N <= ILE_GRAD_MAX_SAMPLES.  Device
 * memory: N * n_window * 4 bytes of scratch when g_Q is requested, and in BF16x3 contexts
 * whenever g_samples, g_Q or lnL_t_out is; a timed-out device wait returns ILE_E_TIMEOUT.
 * flags: ILE_DEVICE_PTRS.
 */
ile_status ile_eval_grad(ile_ctx *ctx, const double *samples, int64_t N, const double *g_lnL, double *g_samples,
                         double *g_Q, double *g_U, double *g_V, double *lnL_t_out, unsigned flags);

/*
 * ln L_marg of Eq. (eq:lnL:MonteCarlo) (result as in ile_integrate, computed with the context's
 * contraction arithmetic) and g_scale times its gradient through lnL_t: the adjoint of
 * ile_eval_grad with g_lnL[n] = g_scale * w_n / sum w.  g_scale: one double (host or device per
 * flags), NULL = 1.  ln_prior and ln_ps enter as constants (their own derivatives are the
 * caller's).  Outputs as in ile_eval_grad; any of them may be NULL.
 */
ile_status ile_integrate_grad(ile_ctx *ctx, const double *samples, const double *ln_prior, const double *ln_ps,
                              int64_t N, const double *g_scale, double *result, double *g_samples, double *g_Q,
                              double *g_U, double *g_V, unsigned flags);

/*
 * The sampler's random-number generator, exposed for known-answer tests: Philox4x32-10 (Salmon,
 * Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), the generator the
 * device sampler draws its words from (Sec. "GPU-accelerated Monte Carlo integration" draws the
 * samples on the GPU).  ctr_key: [n][6] device array, counter words 0..3 then key words 0..1;
 * out: [n][4] device array of output words.  Queued on cuda_stream (a cudaStream_t; NULL = legacy
 * default stream) without waiting; 1 <= n <= 2^24, else ILE_E_ARG.  Allocates nothing.
 */
ile_status ile_philox4x32_10(const uint32_t *ctr_key, int64_t n, uint32_t *out, void *cuda_stream);

/* Wait for the context's stream and return the first device-side error seen since the last call. */
ile_status ile_sync(ile_ctx *ctx);

/*
 * Cap on the device memory this context allocates, in bytes (0 = no cap, the default).  A call
 * that would allocate past the cap returns ILE_E_NOMEM before any device allocation is attempted;
 * the memory the context already holds stays valid and the context stays usable (raise the cap
 * and call again).  For services that must stay within a fixed budget, and for exercising the
 * allocation-failure path.  ile_memory_used reports the bytes the context holds now.
 */
ile_status ile_set_memory_limit(ile_ctx *ctx, size_t bytes);
ile_status ile_memory_used(const ile_ctx *ctx, size_t *bytes);

/*
 * Check of the bounded device-side waits: one block waits on a shared-memory mbarrier phase that
 * nothing completes, with the same bounded sleeping wait the pipelined kernels use, limited to
 * about timeout_s seconds (0 < timeout_s <= 10, else ILE_E_ARG).  The wait gives up, raises the
 * context's timeout flag and the call returns ILE_E_TIMEOUT; the context remains usable.  No
 * fault or trap is involved.
 */
ile_status ile_check_wait_timeout(ile_ctx *ctx, double timeout_s);

/* Human-readable name of a status code (static storage). */
const char *ile_status_string(ile_status st);

/* Last CUDA error message recorded by the context (static storage of the context). */
const char *ile_last_error(const ile_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* ILE_H */
