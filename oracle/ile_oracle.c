/*
 * ile_oracle.c -- plain FP64 CPU oracle for the ILE extrinsic-marginalisation hot path of
 * Wofford et al., "Expanding RIFT" (arXiv:2210.07912).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link, load or call this
 * file: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg use it.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Everything is double precision, written as plain nested loops in the order the paper states
 * the quantities; there is no blocking, fusion or reordering.  Compile with -ffp-contract=off
 * so that every floating-point operation is a separate IEEE operation on every host.
 *
 * Passages followed (section / equation labels of the paper):
 *   - marginal likelihood as a Monte Carlo sum over extrinsic samples: Sec. "Evaluating the
 *     marginalized likelihood", Eq. (eq:lnL:MonteCarlo);
 *   - per-sample likelihood from Q, U, V, antenna factors F_k and spin-weighted harmonics:
 *     App. "Numerical and adaptation approaches needed for strong signals", subsection
 *     "Estimates of signal strength", Eq. (eq:loglikelihood) and Eq. (eq:QUV); the D_ref/D
 *     factor on the data term follows the one-parameter approximation given right after
 *     Eq. (eq:QUV);
 *   - all integrand sums done in log space ("logsumexp"): same appendix, subsection "Choices
 *     for finite-precision floating point arithmetic and overflow";
 *   - adaptive-Cartesian sampler with a separable sampling prior and 100-bin histograms per
 *     adaptive dimension: Sec. "GPU-accelerated Monte Carlo integration";
 *   - n_eff = sum p_k / max p_k: App. "Monte Carlo integration and independent samples",
 *     Eq. (eq:neff); Kish ESS: Eq. (eq:neff_ESS).
 *   - gradient of lnL_t (orc_lnL_t_grad): the chain rule through the same steps; the paper
 *     states no derivative, so this is the exact derivative of the function above (R21).
 *
 * Readings of passages that are silent, garbled or ambiguous:
 *   R1 ln L = Re<h|d> - <h|h>/2 (the first line of Eq. (eq:loglikelihood) is garbled; the
 *      data-only constant is dropped).
 *   R2 the data term carries Re and D_ref/D: h_k = Re[F_k sum_lm Y_lm h_lm] (D_ref/D).
 *   R3 antenna pattern in the textbook wave-frame form (X x Y = -n), GMST an input.
 *   R4 _{-2}Y_lm(iota,phi) = sqrt((2l+1)/4pi) d^l_{m,2}(iota) e^{i m phi} with the explicit
 *      Wigner-d sum d^l_{m'm}; this gives the closed forms common in GW data analysis
 *      (e.g. _{-2}Y_21 = +sqrt(5/16pi) sin(iota)(1+cos(iota)) e^{i phi}).
 *   R5 geocentric reference time, dt_k = -(r_k . n)/c, linear interpolation of Q between bins;
 *      a nearest-sample mode (the sample rint(x), ties to even) serves brute-force cross-checks.
 *   R6 time marginalisation with a uniform prior over the N_t-bin window: LSE_j - ln N_t;
 *      bin j sits at t_c + (j - N_t/2)/f_s.
 *   R7 MC error sigma_I / I with the sample variance s^2/N.
 *   R8 adaptive histogram: likelihood-weighted 100-bin histogram with an eps floor, sampled
 *      through an integer (2^32) cumulative table.
 *   R21 gradient: exact derivative of lnL_t with the interpolation weight differentiated inside
 *      a bin (one-sided at bin edges: the slope of the bin floor(x) lies in); the entries of
 *      Q, U and V are independent real pairs (no Hermitian / symmetric tying of U and V).
 *   R23 rotated network sky frame: pole p along a detector baseline, e1 = z x p normalised,
 *      e2 = p x e1; sampling variables (longitude, sin latitude) in (e1, e2, p).
 *   R22 distance marginalisation: the distance integral sits inside the window sum, i.e. the
 *      marginal of (1/N_t) sum_j exp(a_j x - b x^2) over p(D) prop. to D^2 on [D_min, D_max],
 *      x = D_ref / D, with a_j, b the data and quadratic terms at D = D_ref.
 *   R24 Gaussian-mixture sampler (Sec. "Adaptive sampling with gaussian mixture models" and the
 *      appendix on its implementation), separable form: the sample weight w_n scales the
 *      responsibility in the M-step sums, the mixture weight is divided by sum_n w_n (the
 *      printed E-step cancels w_n), a fixed number of EM steps per iteration started from the
 *      current model, the 1-D Mahalanobis distance |mu_i - mu_j| / sigma in the matching, and the
 *      initial model C equal components evenly spaced over the range with sigma = range / C.
 *   R26 correlated sampling of the sky pair (sampling variables 0 and 1; Sec. "Adaptive sampling
 *      with gaussian mixture models" samples subsets of dimensions jointly, App. "Gaussian mixture
 *      model implementation" gives the multivariate EM, merge and the truncation by rejection):
 *      each component is a bivariate normal truncated to the rectangle, its mass Z_c inside
 *      computed exactly (so ln p_s is the normalised density and the integral stays unbiased);
 *      the component is drawn once per sample and only the whitened pair is redrawn on
 *      rejection (so the accepted density of component c is its truncated normal); the whitening
 *      uses the Cholesky factor of the covariance (any square root gives the same draws' law;
 *      the paper writes the eigen form); floors sigma_j >= 1e-3 of the range, |rho| <= 0.9, the
 *      mean inside the rectangle (after every M-step and merge); the initial model places C
 *      components on the rectangle's diagonal; the cost of a matching is the paper's sum of the
 *      two one-sided Mahalanobis distances of every matched pair.
 *   R25 the M-step mean is clamped into [lo, hi]: a weighted mean of points inside the range lies
 *      inside it, so the clamp changes nothing but rounding excursions at the range ends (the
 *      truncated normals of Sec. "Adaptive sampling with gaussian mixture models" need mu there
 *      for the sampler's tail-safe inverse CDF).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_E_ARG 1
#define ORC_E_RANGE 3
#define ORC_C_SI 299792458.0
#define ORC_PI 3.14159265358979323846

/* One intrinsic point: everything the likelihood needs besides the extrinsic sample. */
typedef struct {
    int n_det;                 /* K */
    int n_modes;               /* M */
    const int *lm;             /* [M][2] (l, m) */
    const double *det_tensor;  /* [K][3][3] */
    const double *det_pos;     /* [K][3], metres, Earth-fixed */
    const double *Q;           /* [K][M][T_ext][2] (re, im) */
    int T_ext;
    double t_start;            /* time of bin 0, seconds, geocentric */
    double fs;                 /* sample rate, Hz */
    const double *U;           /* [K][M][M][2] */
    const double *V;           /* [K][M][M][2] */
    int n_window;              /* N_t */
    double gmst;               /* radians */
    double d_ref;              /* Mpc */
    int nearest;               /* 1: Q at the nearest sample instead of linear interpolation (R5) */
} orc_point;

/* ---------------------------------------------------------------- S1: geometry (R3, R5) */

/* Wave-frame basis X, Y and the unit vector n towards the source, Earth-fixed frame. */
void orc_frame(double ra, double dec, double psi, double gmst, double X[3], double Y[3], double n[3])
{
    double g = gmst - ra;
    double cg = cos(g), sg = sin(g);
    double cd = cos(dec), sd = sin(dec);
    double cp = cos(psi), sp = sin(psi);
    X[0] = -cp * sg - sp * cg * sd;
    X[1] = -cp * cg + sp * sg * sd;
    X[2] = sp * cd;
    Y[0] = sp * sg - cp * cg * sd;
    Y[1] = sp * cg + cp * sg * sd;
    Y[2] = cp * cd;
    n[0] = cd * cg;
    n[1] = -cd * sg;
    n[2] = sd;
}

/* F_+ = sum_ab D_ab (X_a X_b - Y_a Y_b),  F_x = sum_ab D_ab (X_a Y_b + Y_a X_b). */
void orc_antenna(const double *D, double ra, double dec, double psi, double gmst, double out[2])
{
    double X[3], Y[3], n[3];
    orc_frame(ra, dec, psi, gmst, X, Y, n);
    double fp = 0.0, fx = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            fp += D[3 * a + b] * (X[a] * X[b] - Y[a] * Y[b]);
            fx += D[3 * a + b] * (X[a] * Y[b] + Y[a] * X[b]);
        }
    out[0] = fp;
    out[1] = fx;
}

/* Arrival time at the detector minus arrival time at the geocentre. */
double orc_delay(const double *r, double ra, double dec, double gmst)
{
    double X[3], Y[3], n[3];
    orc_frame(ra, dec, 0.0, gmst, X, Y, n);
    return -(r[0] * n[0] + r[1] * n[1] + r[2] * n[2]) / ORC_C_SI;
}

/* ---------------------------------------------------------------- S2: harmonics (R4) */

static double fact(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; i++) f *= (double)i;
    return f;
}

/*
 * Wigner small-d d^l_{m1,m2}(beta) = <l m1| exp(-i beta J_y) |l m2>, explicit sum over k
 * (Wigner's formula; d^l_{m1,m2}(0) = delta_{m1,m2}).
 */
double orc_wigner_d(int l, int m1, int m2, double beta)
{
    double c = cos(0.5 * beta), s = sin(0.5 * beta);
    double pref = sqrt(fact(l + m1) * fact(l - m1) * fact(l + m2) * fact(l - m2));
    double sum = 0.0;
    for (int k = 0; k <= 2 * l; k++) {
        int a = l + m2 - k, b = k, d = l - k - m1, e = k - m2 + m1;
        if (a < 0 || d < 0 || e < 0) continue;
        double sign = ((k - m2 + m1) % 2 == 0) ? 1.0 : -1.0;
        double term = sign / (fact(a) * fact(b) * fact(d) * fact(e));
        term *= pow(c, 2 * l - 2 * k + m2 - m1) * pow(s, 2 * k - m2 + m1);
        sum += term;
    }
    return pref * sum;
}

/* _{-2}Y_lm(iota, phi) = sqrt((2l+1)/4pi) d^l_{m,2}(iota) e^{i m phi}. */
void orc_sylm(int l, int m, double iota, double phi, double out[2])
{
    double amp = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI)) * orc_wigner_d(l, m, 2, iota);
    out[0] = amp * cos(m * phi);
    out[1] = amp * sin(m * phi);
}

/* ---------------------------------------------------------------- S2-S5 per sample */

/* Mode coefficients c_{k,lm} = (D_ref/D) F_k Y_lm and delays for one sample. */
static void coefficients(const orc_point *P, const double th[7], double *c /*[K][M][2]*/, double *dt /*[K]*/)
{
    double ra = th[0], dec = th[1], psi = th[2], iota = th[3], phi = th[4], dist = th[5];
    int K = P->n_det, M = P->n_modes;
    for (int k = 0; k < K; k++) {
        double F[2];
        orc_antenna(P->det_tensor + 9 * k, ra, dec, psi, P->gmst, F);
        dt[k] = orc_delay(P->det_pos + 3 * k, ra, dec, P->gmst);
        for (int a = 0; a < M; a++) {
            double Yv[2];
            orc_sylm(P->lm[2 * a], P->lm[2 * a + 1], iota, phi, Yv);
            double s = P->d_ref / dist;
            c[(k * M + a) * 2 + 0] = s * (F[0] * Yv[0] - F[1] * Yv[1]);
            c[(k * M + a) * 2 + 1] = s * (F[0] * Yv[1] + F[1] * Yv[0]);
        }
    }
}

/* S4: A = 1/4 sum_k [ c^H U_k c + Re(c^T V_k c) ]  ( = <h|h>/2 ). */
static double quadratic(const orc_point *P, const double *c)
{
    int K = P->n_det, M = P->n_modes;
    double A = 0.0;
    for (int k = 0; k < K; k++) {
        const double *ck = c + 2 * k * M;
        const double *Uk = P->U + 2 * (size_t)k * M * M;
        const double *Vk = P->V + 2 * (size_t)k * M * M;
        double u = 0.0, v = 0.0;
        for (int a = 0; a < M; a++)
            for (int b = 0; b < M; b++) {
                double car = ck[2 * a], cai = ck[2 * a + 1];
                double cbr = ck[2 * b], cbi = ck[2 * b + 1];
                double ur = Uk[2 * (a * M + b)], ui = Uk[2 * (a * M + b) + 1];
                double vr = Vk[2 * (a * M + b)], vi = Vk[2 * (a * M + b) + 1];
                /* conj(c_a) U_ab c_b, real part */
                double pr = car * cbr + cai * cbi, pi = car * cbi - cai * cbr; /* conj(c_a) c_b */
                u += pr * ur - pi * ui;
                /* c_a V_ab c_b, real part */
                double qr = car * cbr - cai * cbi, qi = car * cbi + cai * cbr; /* c_a c_b */
                v += qr * vr - qi * vi;
            }
        A += u + v;
    }
    return 0.25 * A;
}

/*
 * lnL(n, j) for every window bin j of one sample (S1-S4), before time marginalisation.
 * data_out[j] (optional) gets the data term alone; *quad_out (optional) gets A.
 * Returns ORC_E_RANGE if any interpolation index leaves [0, T_ext-1].
 */
int orc_lnL_grid(const orc_point *P, const double th[7], double *lnL, double *data_out, double *quad_out)
{
    int K = P->n_det, M = P->n_modes, T = P->T_ext, Nt = P->n_window;
    if (K < 1 || M < 1 || Nt < 1 || T < 2) return ORC_E_ARG;
    double *c = (double *)malloc(sizeof(double) * 2 * K * M);
    double *dt = (double *)malloc(sizeof(double) * K);
    coefficients(P, th, c, dt);
    double A = quadratic(P, c);
    int status = ORC_OK;
    for (int j = 0; j < Nt; j++) {
        double data = 0.0;
        for (int k = 0; k < K; k++) {
            double tau = th[6] + ((double)j - 0.5 * Nt) / P->fs + dt[k];
            double x = (tau - P->t_start) * P->fs;
            /* linear interpolation between samples floor(x) and floor(x) + 1 (reading R5); in the
             * nearest-sample mode the sample closest to x (ties to even), i.e. the interpolation
             * with its weight set to zero at the rounded position */
            double fl = P->nearest ? rint(x) : floor(x);
            double w = P->nearest ? 0.0 : x - fl;
            if (fl < 0.0 || fl + 1.0 > (double)(T - 1)) { status = ORC_E_RANGE; continue; }
            long i = (long)fl;
            for (int a = 0; a < M; a++) {
                const double *q = P->Q + 2 * (((size_t)k * M + a) * T);
                double qr = (1.0 - w) * q[2 * i] + w * q[2 * (i + 1)];
                double qi = (1.0 - w) * q[2 * i + 1] + w * q[2 * (i + 1) + 1];
                double cr = c[2 * (k * M + a)], ci = c[2 * (k * M + a) + 1];
                data += cr * qr + ci * qi; /* Re(conj(c) Q) */
            }
        }
        if (data_out) data_out[j] = data;
        lnL[j] = data - A;
    }
    if (quad_out) *quad_out = A;
    free(c);
    free(dt);
    return status;
}

/* S5: ln L_t = LSE_j lnL(n, j) - ln N_t for one sample. */
static int lnL_t_one(const orc_point *P, const double th[7], double *lnL_grid, double *out)
{
    int st = orc_lnL_grid(P, th, lnL_grid, NULL, NULL);
    int Nt = P->n_window;
    double m = lnL_grid[0];
    for (int j = 1; j < Nt; j++) if (lnL_grid[j] > m) m = lnL_grid[j];
    double s = 0.0;
    for (int j = 0; j < Nt; j++) s += exp(lnL_grid[j] - m);
    *out = m + log(s) - log((double)Nt);
    return st;
}

/* S1-S5 over N samples stored SoA [7][N] (ra, dec, psi, iota, phi, D_Mpc, tc_s). */
int orc_lnL_t(const orc_point *P, const double *samples, long N, double *out, int nthreads)
{
    int status = ORC_OK;
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(| : status)
#endif
    {
        double *grid = (double *)malloc(sizeof(double) * P->n_window);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (long n = 0; n < N; n++) {
            double th[7];
            for (int d = 0; d < 7; d++) th[d] = samples[(size_t)d * N + n];
            status |= lnL_t_one(P, th, grid, out + n);
        }
        free(grid);
    }
    return status;
}

/* ---------------------------------------------------------------- S6: MC integral (R7) */

/*
 * From ln w_n (n < N): ln I = LSE_n ln w_n - ln N; sigma_ln = sigma_I / I with the sample
 * variance; n_eff = sum w / max w; ESS = (sum w)^2 / sum w^2.  Sums are taken relative to the
 * maximum so that no weight overflows.  out = {ln I, sigma_ln, n_eff, ess, max ln w, S1, S2}.
 */
void orc_mc_stats(const double *lnw, long N, double out[7])
{
    double m = -INFINITY;
    for (long n = 0; n < N; n++) if (lnw[n] > m) m = lnw[n];
    double s1 = 0.0, s2 = 0.0;
    for (long n = 0; n < N; n++) {
        double e = exp(lnw[n] - m);
        s1 += e;
        s2 += e * e;
    }
    double Nd = (double)N;
    double mean = s1 / Nd;                       /* in units of e^m */
    double var = (s2 - Nd * mean * mean) / (Nd - 1.0);
    if (var < 0.0) var = 0.0;
    out[0] = m + log(mean);
    out[1] = (N > 1) ? sqrt(var / Nd) / mean : INFINITY;
    out[2] = s1;
    out[3] = s1 * s1 / s2;
    out[4] = m;
    out[5] = s1;
    out[6] = s2;
}

/* ---------------------------------------------------------------- S0: counter-based RNG */

/*
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the Philox S-box on a
 * 128-bit counter with a 64-bit key bumped by the Weyl constants between rounds.
 */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* ---------------------------------------------------------------- S0 / S6: AC sampler (R8) */

#define ORC_NBINS 100
#define ORC_NDIM 7

/*
 * Separable sampling prior over the sampling variables
 *   u0 = ra in [0, 2pi), u1 = sin(dec) in [-1, 1], u2 = psi in [0, pi), u3 = cos(iota) in [-1, 1],
 *   u4 = phi in [0, 2pi), u5 = D in [D_min, D_max] (prior prop. to D^2), u6 = t_c in [-T_c, T_c].
 * A fixed dimension is drawn from its prior; an adaptive one from a 100-bin histogram given by
 * its integer cumulative table cdf[0..100] (cdf[0] = 0, cdf[100] = 2^32).
 */
/* One dimension's Gaussian-mixture sampling prior (App. "Gaussian mixture model
 * implementation", separable form): C components with weights w, means mu, widths sigma, each
 * a normal truncated to the dimension's range; n = samples the model has been trained on. */
#define ORC_GMM_MAX 8
typedef struct {
    int C;
    double w[ORC_GMM_MAX], mu[ORC_GMM_MAX], sigma[ORC_GMM_MAX];
    double n;
} orc_gmm1;

/* The correlated mixture of the sky pair (sampling variables 0 and 1 together; Sec. "Adaptive
 * sampling with gaussian mixture models": correlated sampling in a subset of dimensions; App.
 * "Gaussian mixture model implementation"): C components with weights w, means mu[c] and
 * covariances cov[c] = {S00, S01, S11}, each a bivariate normal truncated to the rectangle
 * [lo0, hi0] x [lo1, hi1]; n = samples the model has been trained on. */
typedef struct {
    int C;
    double w[ORC_GMM_MAX], mu[ORC_GMM_MAX][2], cov[ORC_GMM_MAX][3];
    double n;
} orc_gmm2;

typedef struct {
    double lo[ORC_NDIM], hi[ORC_NDIM];
    int adaptive[ORC_NDIM];
    const uint64_t *cdf; /* [7][101]; rows of fixed dimensions are ignored */
    int sky;             /* 1: variables 0, 1 are (longitude, sin latitude) in the rotated frame */
    double pole[3];      /* Earth-fixed pole of the rotated frame */
    double gmst;
    int gmm[ORC_NDIM];   /* 1: adaptive dimension drawn from its mixture instead of its histogram */
    const orc_gmm1 *model; /* [7] */
    int pair;            /* 1: variables 0 and 1 drawn together from pair_model */
    const orc_gmm2 *pair_model;
} orc_sampler;

/* Standard normal CDF and its inverse (Newton iterations on erfc from a coarse start). */
static double norm_cdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

double orc_norm_ppf(double p)
{
    if (p <= 0.0) return -INFINITY;
    if (p >= 1.0) return INFINITY;
    /* start: logistic approximation, then Newton on Phi(x) - p */
    double x = -log(1.0 / p - 1.0) / 1.702;
    for (int it = 0; it < 100; it++) {
        double f = norm_cdf(x) - p, d = exp(-0.5 * x * x) / sqrt(2.0 * ORC_PI);
        double step = f / d;
        if (step > 2.0) step = 2.0;
        if (step < -2.0) step = -2.0;
        x -= step;
        if (fabs(step) < 1e-15 * (1.0 + fabs(x))) break;
    }
    return x;
}

/* Integer cumulative table of the component weights (2^32 scale, same rule as the histograms). */
void orc_gmm_cum(const orc_gmm1 *g, uint64_t *cw)
{
    double tot = 0.0, acc = 0.0;
    for (int c = 0; c < g->C; c++) tot += g->w[c];
    cw[0] = 0;
    for (int c = 0; c < g->C; c++) {
        acc += g->w[c] / tot;
        if (c + 1 < g->C) {
            double v = floor(acc * 4294967296.0);
            if (v > 4294967296.0) v = 4294967296.0;
            cw[c + 1] = (uint64_t)v;
        }
    }
    cw[g->C] = (uint64_t)1 << 32;
    for (int c = 1; c <= g->C; c++)
        if (cw[c] < cw[c - 1]) cw[c] = cw[c - 1];
}

/* ln of the truncated-mixture density sum_c (w_c / sum w) N(u | mu_c, sigma_c) / Z_c on [lo, hi],
 * Z_c = Phi((hi - mu_c) / sigma_c) - Phi((lo - mu_c) / sigma_c), as a log-sum-exp over c. */
double orc_gmm_lnpdf(const orc_gmm1 *g, double lo, double hi, double u)
{
    double tot = 0.0, l[ORC_GMM_MAX], m = -INFINITY;
    for (int c = 0; c < g->C; c++) tot += g->w[c];
    for (int c = 0; c < g->C; c++) {
        double z = (u - g->mu[c]) / g->sigma[c];
        double Z = norm_cdf((hi - g->mu[c]) / g->sigma[c]) - norm_cdf((lo - g->mu[c]) / g->sigma[c]);
        l[c] = log(g->w[c] / tot) - log(sqrt(2.0 * ORC_PI) * g->sigma[c] * Z) - 0.5 * z * z;
        if (l[c] > m) m = l[c];
    }
    double s = 0.0;
    for (int c = 0; c < g->C; c++) s += exp(l[c] - m);
    return m + log(s);
}

/* Uniform in (0, 1) from the top 23 bits of one 32-bit word. */
static double unit23(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* ---- correlated sky-pair mixture (R26) */

/* Mass of the rectangle [lo0, hi0] x [lo1, hi1] under N(mu, cov): in standardised coordinates
 * u_j = (x_j - mu_j) / sigma_j with correlation rho it is the integral over u_0 in [a_0, b_0] of
 * phi(u_0) [Phi((b_1 - rho u_0) / s) - Phi((a_1 - rho u_0) / s)], s = sqrt(1 - rho^2) (the
 * conditional law of u_1 given u_0), evaluated by composite Simpson over [a_0, b_0] cut to
 * [-12, 12] (4096 panels). */
double orc_bvn_rect(const double mu[2], const double cov[3], const double lo[2], const double hi[2])
{
    double s0 = sqrt(cov[0]), s1 = sqrt(cov[2]);
    double rho = cov[1] / (s0 * s1), s = sqrt(1.0 - rho * rho);
    double a0 = (lo[0] - mu[0]) / s0, b0 = (hi[0] - mu[0]) / s0;
    double a1 = (lo[1] - mu[1]) / s1, b1 = (hi[1] - mu[1]) / s1;
    if (a0 < -12.0) a0 = -12.0;
    if (b0 > 12.0) b0 = 12.0;
    if (!(b0 > a0)) return 0.0;
    const int P = 4096;
    double h = (b0 - a0) / P, sum = 0.0;
    for (int i = 0; i <= P; i++) {
        double u = a0 + i * h;
        double f = exp(-0.5 * u * u) / sqrt(2.0 * ORC_PI) * (norm_cdf((b1 - rho * u) / s) - norm_cdf((a1 - rho * u) / s));
        double wgt = (i == 0 || i == P) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        sum += wgt * f;
    }
    return sum * h / 3.0;
}

/* Every component's mass Z_c inside the rectangle (orc_bvn_rect). */
void orc_gmm2_masses(const orc_gmm2 *g, const double lo[2], const double hi[2], double *Z)
{
    for (int c = 0; c < g->C; c++) Z[c] = orc_bvn_rect(g->mu[c], g->cov[c], lo, hi);
}

/* ln of the truncated pair density sum_c (w_c / sum w) N(x | mu_c, cov_c) / Z_c on the rectangle,
 * Z_c the components' masses (orc_gmm2_masses), as a log-sum-exp over c. */
double orc_gmm2_lnpdf_z(const orc_gmm2 *g, const double *Z, const double x[2])
{
    double tot = 0.0, l[ORC_GMM_MAX], m = -INFINITY;
    for (int c = 0; c < g->C; c++) tot += g->w[c];
    for (int c = 0; c < g->C; c++) {
        const double *S = g->cov[c];
        double det = S[0] * S[2] - S[1] * S[1];
        double d0 = x[0] - g->mu[c][0], d1 = x[1] - g->mu[c][1];
        double q = (S[2] * d0 * d0 - 2.0 * S[1] * d0 * d1 + S[0] * d1 * d1) / det;
        l[c] = log(g->w[c] / tot) - log(2.0 * ORC_PI * sqrt(det) * Z[c]) - 0.5 * q;
        if (l[c] > m) m = l[c];
    }
    double sum = 0.0;
    for (int c = 0; c < g->C; c++) sum += exp(l[c] - m);
    return m + log(sum);
}

double orc_gmm2_lnpdf(const orc_gmm2 *g, const double lo[2], const double hi[2], const double x[2])
{
    double Z[ORC_GMM_MAX];
    orc_gmm2_masses(g, lo, hi, Z);
    return orc_gmm2_lnpdf_z(g, Z, x);
}

/* Integer cumulative table of mixture weights w[0..C-1] (2^32 scale, same rule as the histograms). */
static void weights_cum(const double *w, int C, uint64_t *cw)
{
    double tot = 0.0, acc = 0.0;
    for (int c = 0; c < C; c++) tot += w[c];
    cw[0] = 0;
    for (int c = 0; c < C; c++) {
        acc += w[c] / tot;
        if (c + 1 < C) {
            double v = floor(acc * 4294967296.0);
            if (v > 4294967296.0) v = 4294967296.0;
            cw[c + 1] = (uint64_t)v;
        }
    }
    cw[C] = (uint64_t)1 << 32;
    for (int c = 1; c <= C; c++)
        if (cw[c] < cw[c - 1]) cw[c] = cw[c - 1];
}

/* Square root L (lower triangular, L L^T = cov) of component c and the box [blo, bhi] of whitened
 * coordinates y = L^-1 (x - mu) that contains the image of the rectangle (its corners' extent). */
static void pair_whiten(const orc_gmm2 *g, int c, const double lo[2], const double hi[2], double L[3],
                        double blo[2], double bhi[2])
{
    const double *S = g->cov[c];
    L[0] = sqrt(S[0]);
    L[1] = S[1] / L[0];
    L[2] = sqrt(S[2] - L[1] * L[1]);
    blo[0] = blo[1] = INFINITY;
    bhi[0] = bhi[1] = -INFINITY;
    for (int k = 0; k < 4; k++) {
        double x0 = (k & 1) ? hi[0] : lo[0], x1 = (k & 2) ? hi[1] : lo[1];
        double y0 = (x0 - g->mu[c][0]) / L[0];
        double y1 = (x1 - g->mu[c][1] - L[1] * y0) / L[2];
        if (y0 < blo[0]) blo[0] = y0;
        if (y0 > bhi[0]) bhi[0] = y0;
        if (y1 < blo[1]) blo[1] = y1;
        if (y1 > bhi[1]) bhi[1] = y1;
    }
}

/* One draw of the pair for sample n: the component is the largest c with cw[c] <= a; then, for
 * attempt t = 0, 1, ..., the Philox block 4 + t gives two words v_0, v_1, the whitened pair is
 * y_j = Phi^-1(Phi(blo_j) + v_j (Phi(bhi_j) - Phi(blo_j))) (standard normals truncated to the box)
 * and x = mu_c + L_c y; the first x inside the rectangle is kept (at most 1024 attempts; returns
 * the attempt count, or -1).  The accepted x has density N(x | mu_c, cov_c) / Z_c on the rectangle. */
int orc_pair_draw(const orc_gmm2 *g, const double lo[2], const double hi[2], uint32_t a, const uint32_t ctr0[3],
                  const uint32_t key[2], double x[2], int *comp)
{
    uint64_t cw[ORC_GMM_MAX + 1];
    weights_cum(g->w, g->C, cw);
    int c = 0;
    for (int j = 1; j < g->C; j++)
        if (cw[j] <= (uint64_t)a) c = j;
    *comp = c;
    double L[3], blo[2], bhi[2];
    pair_whiten(g, c, lo, hi, L, blo, bhi);
    for (int t = 0; t < 1024; t++) {
        uint32_t ctr[4] = {ctr0[0], ctr0[1], ctr0[2], 4u + (uint32_t)t}, w[4];
        orc_philox4x32_10(ctr, key, w);
        double y[2];
        for (int j = 0; j < 2; j++) {
            double P1 = norm_cdf(blo[j]), P2 = norm_cdf(bhi[j]);
            y[j] = orc_norm_ppf(P1 + unit23(w[j]) * (P2 - P1));
        }
        x[0] = g->mu[c][0] + L[0] * y[0];
        x[1] = g->mu[c][1] + L[1] * y[0] + L[2] * y[1];
        if (x[0] >= lo[0] && x[0] <= hi[0] && x[1] >= lo[1] && x[1] <= hi[1]) return t + 1;
    }
    return -1;
}

/* Floors that keep every pair component usable by the sampler: sigma_j >= 1e-3 (hi_j - lo_j),
 * |rho| <= 0.9, the mean inside the rectangle. */
static void pair_floor(orc_gmm2 *g, int c, const double lo[2], const double hi[2])
{
    double *S = g->cov[c];
    for (int j = 0; j < 2; j++) {
        double smin = 1e-3 * (hi[j] - lo[j]);
        if (S[2 * j] < smin * smin) S[2 * j] = smin * smin;
        if (g->mu[c][j] < lo[j]) g->mu[c][j] = lo[j];
        if (g->mu[c][j] > hi[j]) g->mu[c][j] = hi[j];
    }
    double lim = 0.9 * sqrt(S[0] * S[2]);
    if (S[1] > lim) S[1] = lim;
    if (S[1] < -lim) S[1] = -lim;
}

/*
 * One EM step of the pair on the batch (points x_n = (u0_n, u1_n), sample weights w_n), the
 * multivariate form of App. "Gaussian mixture model implementation" with the sample weight in the
 * sums (R24): r_nc prop. to w_c N(x_n | mu_c, cov_c) (untruncated), S0_c = sum w_n r_nc,
 * mu_c = sum w_n r_nc x_n / S0_c, cov_c = sum w_n r_nc (x_n - mu_c)(x_n - mu_c)^T / S0_c,
 * w_c = S0_c / sum w_n; then the floors; a component with S0_c <= 1e-12 sum w keeps its
 * parameters with weight 1e-3; weights renormalised.
 */
void orc_gmm2_em_step(const double *u0, const double *u1, const double *wn, long N, orc_gmm2 *g, const double lo[2],
                      const double hi[2])
{
    double S0[ORC_GMM_MAX] = {0}, S1[ORC_GMM_MAX][2] = {{0}}, S2[ORC_GMM_MAX][3] = {{0}}, W = 0.0;
    for (long n = 0; n < N; n++) {
        double l[ORC_GMM_MAX], m = -INFINITY, tot = 0.0;
        for (int c = 0; c < g->C; c++) {
            const double *S = g->cov[c];
            double det = S[0] * S[2] - S[1] * S[1];
            double d0 = u0[n] - g->mu[c][0], d1 = u1[n] - g->mu[c][1];
            double q = (S[2] * d0 * d0 - 2.0 * S[1] * d0 * d1 + S[0] * d1 * d1) / det;
            l[c] = log(g->w[c]) - 0.5 * log(det) - 0.5 * q;
            if (l[c] > m) m = l[c];
        }
        for (int c = 0; c < g->C; c++) {
            l[c] = exp(l[c] - m);
            tot += l[c];
        }
        W += wn[n];
        for (int c = 0; c < g->C; c++) {
            double q = wn[n] * l[c] / tot;
            S0[c] += q;
            S1[c][0] += q * u0[n];
            S1[c][1] += q * u1[n];
            S2[c][0] += q * u0[n] * u0[n];
            S2[c][1] += q * u0[n] * u1[n];
            S2[c][2] += q * u1[n] * u1[n];
        }
    }
    double wsum = 0.0;
    for (int c = 0; c < g->C; c++) {
        if (S0[c] > 1e-12 * W) {
            double m0 = S1[c][0] / S0[c], m1 = S1[c][1] / S0[c];
            g->mu[c][0] = m0;
            g->mu[c][1] = m1;
            g->cov[c][0] = S2[c][0] / S0[c] - m0 * m0;
            g->cov[c][1] = S2[c][1] / S0[c] - m0 * m1;
            g->cov[c][2] = S2[c][2] / S0[c] - m1 * m1;
            pair_floor(g, c, lo, hi);
            g->w[c] = S0[c] / W;
        } else {
            g->w[c] = 1e-3;
        }
        wsum += g->w[c];
    }
    for (int c = 0; c < g->C; c++) g->w[c] /= wsum;
}

/* Mahalanobis distance of d under covariance S: sqrt(d^T S^-1 d). */
static double mahalanobis(const double d[2], const double S[3])
{
    double det = S[0] * S[2] - S[1] * S[1];
    return sqrt((S[2] * d[0] * d[0] - 2.0 * S[1] * d[0] * d[1] + S[0] * d[1] * d[1]) / det);
}

/* Online merge of the batch pair model into the current one (App. "Gaussian mixture model
 * implementation"): the permutation matching batch component i to current component j with the
 * least sum of sqrt((mu_j - mu_i)^T S_i^-1 (mu_j - mu_i)) + sqrt((mu_i - mu_j)^T S_j^-1 (mu_i - mu_j))
 * (first such in lexicographic order), then mu = (N w_j mu_j + M w_i mu_i) / (N w_j + M w_i),
 * S = (N w_j S_j + M w_i S_i) / (...) + (N w_j mu_j mu_j^T + M w_i mu_i mu_i^T) / (...) - mu mu^T,
 * w = (N w_j + M w_i) / (N + M), then the floors; n <- N + M. */
void orc_gmm2_merge(const orc_gmm2 *cur, const orc_gmm2 *bat, double M, const double lo[2], const double hi[2],
                    orc_gmm2 *out)
{
    const int C = cur->C;
    int perm[ORC_GMM_MAX], best[ORC_GMM_MAX];
    for (int i = 0; i < C; i++) perm[i] = best[i] = i;
    double best_cost = INFINITY;
    for (;;) {
        double cost = 0.0;
        for (int a = 0; a < C; a++) {
            int j = perm[a];
            double d[2] = {cur->mu[j][0] - bat->mu[a][0], cur->mu[j][1] - bat->mu[a][1]};
            cost += mahalanobis(d, bat->cov[a]) + mahalanobis(d, cur->cov[j]);
        }
        if (cost < best_cost) {
            best_cost = cost;
            for (int a = 0; a < C; a++) best[a] = perm[a];
        }
        int i = C - 2;
        while (i >= 0 && perm[i] > perm[i + 1]) i--;
        if (i < 0) break;
        int j = C - 1;
        while (perm[j] < perm[i]) j--;
        int t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
        for (int x = i + 1, y = C - 1; x < y; x++, y--) {
            t = perm[x];
            perm[x] = perm[y];
            perm[y] = t;
        }
    }
    const double N = cur->n;
    out->C = C;
    for (int a = 0; a < C; a++) {
        int j = best[a];
        double A = N * cur->w[j], B = M * bat->w[a];
        double m0 = (A * cur->mu[j][0] + B * bat->mu[a][0]) / (A + B);
        double m1 = (A * cur->mu[j][1] + B * bat->mu[a][1]) / (A + B);
        out->mu[a][0] = m0;
        out->mu[a][1] = m1;
        out->cov[a][0] = (A * cur->cov[j][0] + B * bat->cov[a][0]) / (A + B) +
                         (A * cur->mu[j][0] * cur->mu[j][0] + B * bat->mu[a][0] * bat->mu[a][0]) / (A + B) - m0 * m0;
        out->cov[a][1] = (A * cur->cov[j][1] + B * bat->cov[a][1]) / (A + B) +
                         (A * cur->mu[j][0] * cur->mu[j][1] + B * bat->mu[a][0] * bat->mu[a][1]) / (A + B) - m0 * m1;
        out->cov[a][2] = (A * cur->cov[j][2] + B * bat->cov[a][2]) / (A + B) +
                         (A * cur->mu[j][1] * cur->mu[j][1] + B * bat->mu[a][1] * bat->mu[a][1]) / (A + B) - m1 * m1;
        out->w[a] = (A + B) / (N + M);
        pair_floor(out, a, lo, hi);
    }
    out->n = N + M;
}

/* Initial pair model: C equal components with means on the rectangle's diagonal at the centres
 * of C equal slices, standard deviations (hi_j - lo_j) / C, no correlation, trained on no samples. */
void orc_gmm2_init(orc_gmm2 *g, int C, const double lo[2], const double hi[2])
{
    g->C = C;
    for (int c = 0; c < C; c++) {
        g->w[c] = 1.0 / C;
        for (int j = 0; j < 2; j++) g->mu[c][j] = lo[j] + (c + 0.5) * (hi[j] - lo[j]) / C;
        g->cov[c][0] = ((hi[0] - lo[0]) / C) * ((hi[0] - lo[0]) / C);
        g->cov[c][1] = 0.0;
        g->cov[c][2] = ((hi[1] - lo[1]) / C) * ((hi[1] - lo[1]) / C);
    }
    g->n = 0.0;
}

void orc_gmm2_update(orc_gmm2 *g, const double *u0, const double *u1, const double *wn, long N, int iters,
                     const double lo[2], const double hi[2])
{
    orc_gmm2 bat = *g, out;
    for (int it = 0; it < iters; it++) orc_gmm2_em_step(u0, u1, wn, N, &bat, lo, hi);
    orc_gmm2_merge(g, &bat, (double)N, lo, hi, &out);
    *g = out;
}

/* Rotated network-frame sky (R23): orthonormal (e1, e2, p) with p = pole / |pole|,
 * e1 = (z x p) / |z x p| (x when p is along z), e2 = p x e1. */
void orc_sky_frame(const double pole[3], double e1[3], double e2[3], double p[3])
{
    double n = sqrt(pole[0] * pole[0] + pole[1] * pole[1] + pole[2] * pole[2]);
    for (int i = 0; i < 3; i++) p[i] = pole[i] / n;
    e1[0] = -p[1];
    e1[1] = p[0];
    e1[2] = 0.0;
    double m = sqrt(e1[0] * e1[0] + e1[1] * e1[1]);
    if (m < 1e-6) {
        e1[0] = 1.0;
        e1[1] = 0.0;
    } else {
        e1[0] /= m;
        e1[1] /= m;
    }
    e2[0] = p[1] * e1[2] - p[2] * e1[1];
    e2[1] = p[2] * e1[0] - p[0] * e1[2];
    e2[2] = p[0] * e1[1] - p[1] * e1[0];
}

/* Prior density of sampling variable d at u. */
static double ln_prior(const orc_sampler *S, int d, double u)
{
    double lo = S->lo[d], hi = S->hi[d];
    if (d == 5) return log(3.0 * u * u / (hi * hi * hi - lo * lo * lo));
    return -log(hi - lo);
}

/*
 * Draw samples n0 .. n0+N-1 of iteration `iter` of point `point`.  Words: Philox4x32-10 with
 * key (seed_lo, seed_hi) and counter (n, iter, point, block), block = 0..3 -> 16 words; sampling
 * variable d uses words 2d and 2d+1.  Writes the physical parameters SoA [7][N], ln p - ln p_s,
 * and the bin of every adaptive dimension ([7][N], 255 for fixed ones).
 */
void orc_sample(const orc_sampler *S, uint64_t seed, uint32_t iter, uint32_t point, long n0, long N,
                double *theta, double *lnp_minus_lnps, uint8_t *bins, double *u_out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double pair_lo[2] = {S->lo[0], S->lo[1]}, pair_hi[2] = {S->hi[0], S->hi[1]}, pair_Z[ORC_GMM_MAX];
    if (S->pair) orc_gmm2_masses(S->pair_model, pair_lo, pair_hi, pair_Z);
    for (long s = 0; s < N; s++) {
        uint32_t n = (uint32_t)(n0 + s);
        uint32_t words[16];
        for (uint32_t blk = 0; blk < 4; blk++) {
            uint32_t ctr[4] = {n, iter, point, blk};
            orc_philox4x32_10(ctr, key, words + 4 * blk);
        }
        double lw = 0.0;
        double pair_x[2] = {0.0, 0.0};
        int pair_c = 0;
        if (S->pair) {
            /* the sky pair together (R26); its component uses word 0, its attempts Philox blocks 4.. */
            uint32_t ctr0[3] = {n, iter, point};
            if (orc_pair_draw(S->pair_model, pair_lo, pair_hi, words[0], ctr0, key, pair_x, &pair_c) < 0) {
                pair_x[0] = 0.5 * (pair_lo[0] + pair_hi[0]);
                pair_x[1] = 0.5 * (pair_lo[1] + pair_hi[1]);
            }
            lw += ln_prior(S, 0, pair_x[0]) + ln_prior(S, 1, pair_x[1]) - orc_gmm2_lnpdf_z(S->pair_model, pair_Z, pair_x);
        }
        for (int d = 0; d < ORC_NDIM; d++) {
            double lo = S->lo[d], hi = S->hi[d], u;
            uint32_t a = words[2 * d], b = words[2 * d + 1];
            int bin = 255;
            if (S->pair && d < 2) {
                u = pair_x[d];
                bin = pair_c;
            } else if (S->adaptive[d] && S->gmm[d]) {
                /* mixture: component = largest c with cw[c] <= a; inside it, the truncated normal
                 * by inverting its CDF at Phi(a_c) + v (Phi(b_c) - Phi(a_c)) */
                const orc_gmm1 *g = S->model + d;
                uint64_t cw[ORC_GMM_MAX + 1];
                orc_gmm_cum(g, cw);
                bin = 0;
                for (int c = 0; c < g->C; c++)
                    if (cw[c] <= (uint64_t)a) bin = c;
                double Pa = norm_cdf((lo - g->mu[bin]) / g->sigma[bin]);
                double Pb = norm_cdf((hi - g->mu[bin]) / g->sigma[bin]);
                u = g->mu[bin] + g->sigma[bin] * orc_norm_ppf(Pa + unit23(b) * (Pb - Pa));
                if (u < lo) u = lo;
                if (u > hi) u = hi;
                lw += ln_prior(S, d, u) - orc_gmm_lnpdf(g, lo, hi, u);
            } else if (S->adaptive[d]) {
                const uint64_t *cdf = S->cdf + (size_t)d * (ORC_NBINS + 1);
                bin = 0;
                for (int q = 0; q < ORC_NBINS; q++)
                    if (cdf[q] <= (uint64_t)a) bin = q; /* largest q with cdf[q] <= a */
                double width = (hi - lo) / ORC_NBINS;
                u = lo + ((double)bin + unit23(b)) * width;
                double mass = (double)(cdf[bin + 1] - cdf[bin]) / 4294967296.0;
                lw += ln_prior(S, d, u) - (log(mass) - log(width));
            } else {
                double v = unit23(a);
                if (d == 5)
                    u = cbrt(lo * lo * lo + v * (hi * hi * hi - lo * lo * lo));
                else
                    u = lo + v * (hi - lo);
            }
            double phys = u;
            if (d == 1) phys = asin(u);
            if (d == 3) phys = acos(u);
            if (S->sky && d == 1) {
                /* (longitude, latitude) in the rotated frame -> Earth-fixed direction -> (ra, dec) */
                double e1[3], e2[3], p[3], nv[3], lon = theta[s], lat = phys;
                orc_sky_frame(S->pole, e1, e2, p);
                for (int i = 0; i < 3; i++) nv[i] = cos(lat) * cos(lon) * e1[i] + cos(lat) * sin(lon) * e2[i] + sin(lat) * p[i];
                double ra = S->gmst - atan2(-nv[1], nv[0]);
                ra -= 2.0 * ORC_PI * floor(ra / (2.0 * ORC_PI));
                theta[s] = ra;
                phys = asin(nv[2]);
            }
            theta[(size_t)d * N + s] = phys;
            bins[(size_t)d * N + s] = (uint8_t)bin;
            if (u_out) u_out[(size_t)d * N + s] = u;
        }
        lnp_minus_lnps[s] = lw;
    }
}

/*
 * Weighted histogram of one adaptive dimension: h_b = sum over samples in bin b of w_n / sum w,
 * with w_n = exp(ln w_n - max ln w).  hist gets 100 values.
 */
void orc_hist(const double *lnw, const uint8_t *bin, long N, double *hist)
{
    double m = -INFINITY;
    for (long n = 0; n < N; n++) if (lnw[n] > m) m = lnw[n];
    double tot = 0.0;
    for (int b = 0; b < ORC_NBINS; b++) hist[b] = 0.0;
    for (long n = 0; n < N; n++) {
        double e = exp(lnw[n] - m);
        hist[bin[n]] += e;
        tot += e;
    }
    for (int b = 0; b < ORC_NBINS; b++) hist[b] /= tot;
}

/*
 * New sampling pdf of one adaptive dimension from its histogram sums h (any positive scale):
 * bin mass (1 - eps) h_b / sum h + eps / 100, accumulated left to right in FP64 and cut to the
 * integer table cdf[b] = floor(2^32 * sum_{b' < b} mass_b'), cdf[0] = 0, cdf[100] = 2^32.
 */
void orc_cdf_from_hist(const double *h, double eps, uint64_t *cdf)
{
    double tot = 0.0;
    for (int b = 0; b < ORC_NBINS; b++) tot += h[b];
    double acc = 0.0;
    cdf[0] = 0;
    for (int b = 0; b < ORC_NBINS; b++) {
        double mass = (1.0 - eps) * (h[b] / tot) + eps / ORC_NBINS;
        acc += mass;
        if (b + 1 < ORC_NBINS) {
            double v = floor(acc * 4294967296.0);
            if (v > 4294967296.0) v = 4294967296.0;
            cdf[b + 1] = (uint64_t)v;
        }
    }
    cdf[ORC_NBINS] = (uint64_t)1 << 32;
    for (int b = 1; b <= ORC_NBINS; b++)
        if (cdf[b] < cdf[b - 1]) cdf[b] = cdf[b - 1];
}

/* Uniform table: every bin 2^32 / 100 (the last bin takes the remainder). */
void orc_cdf_uniform(uint64_t *cdf)
{
    for (int b = 0; b < ORC_NBINS; b++) cdf[b] = ((uint64_t)b << 32) / ORC_NBINS;
    cdf[ORC_NBINS] = (uint64_t)1 << 32;
}

int orc_version(void) { return 1; }

/*
 * One adaptive update of a dimension's mixture (App. "Gaussian mixture model implementation"):
 * `iters` EM steps on the batch (samples u_n with weights w_n, starting from the current model),
 * then the online merge of the batch model into the current one.
 *   E-step: r_nc = w_c N(u_n | mu_c, sigma_c) / sum_c' (...)   (untruncated normal densities)
 *   M-step: S0_c = sum_n w_n r_nc, mu_c = sum_n w_n r_nc u_n / S0_c,
 *           sigma_c^2 = sum_n w_n r_nc (u_n - mu_c)^2 / S0_c, w_c = S0_c / sum_n w_n
 *   (sigma_c >= (hi - lo) 1e-3; a component with S0_c <= 1e-12 sum w keeps its parameters, with
 *   weight 1e-3; weights are renormalised)
 *   merge: match each batch component i to a current component j (a permutation) minimising
 *   sum |mu_i - mu_j| (1/sigma_i + 1/sigma_j) (the 1-D Mahalanobis distances both ways), then
 *   combine with N = current model's sample count, M = batch size:
 *   mu = (N w_j mu_j + M w_i mu_i) / (N w_j + M w_i),
 *   sigma^2 = (N w_j sigma_j^2 + M w_i sigma_i^2) / (...) + (N w_j mu_j^2 + M w_i mu_i^2) / (...) - mu^2,
 *   w = (N w_j + M w_i) / (N + M); n <- N + M.
 */
void orc_gmm_em_step(const double *u, const double *wn, long N, orc_gmm1 *g, double lo, double hi)
{
    double S0[ORC_GMM_MAX] = {0}, S1[ORC_GMM_MAX] = {0}, S2[ORC_GMM_MAX] = {0}, W = 0.0;
    for (long n = 0; n < N; n++) {
        /* r_c prop. to w_c N(u | mu_c, sigma_c), scaled by the largest term before exponentiating */
        double r[ORC_GMM_MAX], l[ORC_GMM_MAX], m = -INFINITY, tot = 0.0;
        for (int c = 0; c < g->C; c++) {
            double z = (u[n] - g->mu[c]) / g->sigma[c];
            l[c] = log(g->w[c] / g->sigma[c]) - 0.5 * z * z;
            if (l[c] > m) m = l[c];
        }
        for (int c = 0; c < g->C; c++) {
            r[c] = exp(l[c] - m);
            tot += r[c];
        }
        W += wn[n];
        for (int c = 0; c < g->C; c++) {
            double q = wn[n] * r[c] / tot;
            S0[c] += q;
            S1[c] += q * u[n];
            S2[c] += q * u[n] * u[n];
        }
    }
    double smin = (hi - lo) * 1e-3, wsum = 0.0;
    for (int c = 0; c < g->C; c++) {
        if (S0[c] > 1e-12 * W) {
            double mu = S1[c] / S0[c], var = S2[c] / S0[c] - mu * mu;
            g->mu[c] = mu < lo ? lo : (mu > hi ? hi : mu); /* R25: a weighted mean of points in range */
            g->sigma[c] = sqrt(var > smin * smin ? var : smin * smin);
            g->w[c] = S0[c] / W;
        } else {
            g->w[c] = 1e-3;
        }
        wsum += g->w[c];
    }
    for (int c = 0; c < g->C; c++) g->w[c] /= wsum;
}

void orc_gmm_merge(const orc_gmm1 *cur, const orc_gmm1 *bat, double M, orc_gmm1 *out)
{
    const int C = cur->C;
    int perm[ORC_GMM_MAX], best[ORC_GMM_MAX];
    for (int i = 0; i < C; i++) perm[i] = best[i] = i;
    double best_cost = INFINITY;
    /* every permutation in lexicographic order; the first one of least cost is kept */
    for (;;) {
        double cost = 0.0;
        for (int a = 0; a < C; a++) {
            int j = perm[a];
            cost += fabs(cur->mu[j] - bat->mu[a]) / bat->sigma[a] + fabs(bat->mu[a] - cur->mu[j]) / cur->sigma[j];
        }
        if (cost < best_cost) {
            best_cost = cost;
            for (int a = 0; a < C; a++) best[a] = perm[a];
        }
        /* next permutation */
        int i = C - 2;
        while (i >= 0 && perm[i] > perm[i + 1]) i--;
        if (i < 0) break;
        int j = C - 1;
        while (perm[j] < perm[i]) j--;
        int t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
        for (int x = i + 1, y = C - 1; x < y; x++, y--) {
            t = perm[x];
            perm[x] = perm[y];
            perm[y] = t;
        }
    }
    const double N = cur->n;
    out->C = C;
    for (int a = 0; a < C; a++) {
        int j = best[a];
        double A = N * cur->w[j], B = M * bat->w[a];
        double mu = (A * cur->mu[j] + B * bat->mu[a]) / (A + B);
        double var = (A * cur->sigma[j] * cur->sigma[j] + B * bat->sigma[a] * bat->sigma[a]) / (A + B) +
                     (A * cur->mu[j] * cur->mu[j] + B * bat->mu[a] * bat->mu[a]) / (A + B) - mu * mu;
        out->mu[a] = mu;
        out->sigma[a] = sqrt(var > 0.0 ? var : 0.0);
        out->w[a] = (A + B) / (N + M);
    }
    out->n = N + M;
}

/* Initial model: C equal components, means at the centres of C equal slices of [lo, hi],
 * sigma = (hi - lo) / C, trained on no samples (so the first merge keeps the batch model). */
void orc_gmm_init(orc_gmm1 *g, int C, double lo, double hi)
{
    g->C = C;
    for (int c = 0; c < C; c++) {
        g->w[c] = 1.0 / C;
        g->mu[c] = lo + (c + 0.5) * (hi - lo) / C;
        g->sigma[c] = (hi - lo) / C;
    }
    g->n = 0.0;
}

void orc_gmm_update(orc_gmm1 *g, const double *u, const double *wn, long N, int iters, double lo, double hi)
{
    orc_gmm1 bat = *g, out;
    for (int it = 0; it < iters; it++) orc_gmm_em_step(u, wn, N, &bat, lo, hi);
    orc_gmm_merge(g, &bat, (double)N, &out);
    *g = out;
}

/* ---------------------------------------------------------------- gradients (adjoint checks) */

/* d/dbeta of the Wigner small-d d^l_{m1,m2}(beta), term by term of the explicit sum. */
double orc_wigner_d_deriv(int l, int m1, int m2, double beta)
{
    double c = cos(0.5 * beta), s = sin(0.5 * beta);
    double pref = sqrt(fact(l + m1) * fact(l - m1) * fact(l + m2) * fact(l - m2));
    double sum = 0.0;
    for (int k = 0; k <= 2 * l; k++) {
        int a = l + m2 - k, b = k, d = l - k - m1, e = k - m2 + m1;
        if (a < 0 || d < 0 || e < 0) continue;
        double sign = ((k - m2 + m1) % 2 == 0) ? 1.0 : -1.0;
        double coef = sign / (fact(a) * fact(b) * fact(d) * fact(e));
        int P = 2 * l - 2 * k + m2 - m1, S = 2 * k - m2 + m1;
        /* d/dbeta c^P s^S = (1/2) (S c^(P+1) s^(S-1) - P c^(P-1) s^(S+1)) */
        double t = 0.0;
        if (S > 0) t += S * pow(c, P + 1) * pow(s, S - 1);
        if (P > 0) t -= P * pow(c, P - 1) * pow(s, S + 1);
        sum += coef * 0.5 * t;
    }
    return pref * sum;
}

/*
 * Gradient of lnL_t(theta) (time-marginalised, Eq. (eq:loglikelihood) with the window LSE) for
 * one sample, times the upstream gradient g:
 *   g_th[7]  += g d lnL_t / d(ra, dec, psi, iota, phi, D, t_c)
 *   gQ       += g d lnL_t / d(Re Q, Im Q)   [K][M][T_ext][2]   (may be NULL)
 *   gU, gV   += g d lnL_t / d(Re, Im) of every entry, the entries taken as independent reals
 *               [K][M][M][2]   (may be NULL)
 * lnL_t = LSE_j lnL(j) - ln N_t, so d lnL_t = sum_j pi_j d lnL(j) with pi the softmax over j.
 * Derivatives: c_ka = (D_ref/D) F_k Y_a; F through the wave frame (X, Y) of (ra, dec, psi);
 * Y through d^l_{m,2}(iota) e^{i m phi}; the window position through t_c and the delays
 * dt_k(ra, dec) (the linear interpolation gives the slope Q[i+1] - Q[i]).
 */
int orc_lnL_t_grad(const orc_point *P, const double th[7], double g, double *g_th, double *gQ, double *gU,
                   double *gV, double *lnL_t_out)
{
    int K = P->n_det, M = P->n_modes, T = P->T_ext, Nt = P->n_window;
    double ra = th[0], dec = th[1], psi = th[2], iota = th[3], phi = th[4], dist = th[5], tc = th[6];
    double sD = P->d_ref / dist;
    /* frame and its derivatives: X = cos(psi) a + sin(psi) b, Y = -sin(psi) a + cos(psi) b */
    double gh = P->gmst - ra, cg = cos(gh), sg = sin(gh), cd = cos(dec), sd = sin(dec), cp = cos(psi), sp = sin(psi);
    double av[3] = {-sg, -cg, 0.0}, bv[3] = {-cg * sd, sg * sd, cd};
    double da_dg[3] = {-cg, sg, 0.0}, db_dg[3] = {sg * sd, cg * sd, 0.0}, db_dd[3] = {-cg * cd, sg * cd, -sd};
    double X[3], Y[3], dX[3][3], dY[3][3]; /* dX[p] = dX/d(ra, dec, psi) */
    for (int q = 0; q < 3; q++) {
        X[q] = cp * av[q] + sp * bv[q];
        Y[q] = -sp * av[q] + cp * bv[q];
        /* d/d ra = -d/dg */
        dX[0][q] = -(cp * da_dg[q] + sp * db_dg[q]);
        dY[0][q] = -(-sp * da_dg[q] + cp * db_dg[q]);
        dX[1][q] = sp * db_dd[q];
        dY[1][q] = cp * db_dd[q];
        dX[2][q] = Y[q];
        dY[2][q] = -X[q];
    }
    double nv[3] = {cd * cg, -cd * sg, sd};
    double dn[2][3] = {{cd * sg, cd * cg, 0.0}, {-sd * cg, sd * sg, cd}}; /* d n / d(ra, dec) */
    double *F = (double *)malloc(sizeof(double) * 2 * K), *dF = (double *)malloc(sizeof(double) * 2 * K * 3);
    double *dt = (double *)malloc(sizeof(double) * K), *ddt = (double *)malloc(sizeof(double) * K * 2);
    for (int k = 0; k < K; k++) {
        const double *D = P->det_tensor + 9 * k;
        double fp = 0, fx = 0;
        double dfp[3] = {0, 0, 0}, dfx[3] = {0, 0, 0};
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double Dab = D[3 * a + b];
                fp += Dab * (X[a] * X[b] - Y[a] * Y[b]);
                fx += Dab * (X[a] * Y[b] + Y[a] * X[b]);
                for (int p = 0; p < 3; p++) {
                    dfp[p] += Dab * (dX[p][a] * X[b] + X[a] * dX[p][b] - dY[p][a] * Y[b] - Y[a] * dY[p][b]);
                    dfx[p] += Dab * (dX[p][a] * Y[b] + X[a] * dY[p][b] + dY[p][a] * X[b] + Y[a] * dX[p][b]);
                }
            }
        F[2 * k] = fp;
        F[2 * k + 1] = fx;
        for (int p = 0; p < 3; p++) {
            dF[(k * 3 + p) * 2] = dfp[p];
            dF[(k * 3 + p) * 2 + 1] = dfx[p];
        }
        const double *r = P->det_pos + 3 * k;
        dt[k] = -(r[0] * nv[0] + r[1] * nv[1] + r[2] * nv[2]) / ORC_C_SI;
        for (int p = 0; p < 2; p++) ddt[2 * k + p] = -(r[0] * dn[p][0] + r[1] * dn[p][1] + r[2] * dn[p][2]) / ORC_C_SI;
    }
    /* harmonics and their iota derivative */
    double *y = (double *)malloc(sizeof(double) * 2 * M), *dy = (double *)malloc(sizeof(double) * 2 * M);
    for (int a = 0; a < M; a++) {
        int l = P->lm[2 * a], m = P->lm[2 * a + 1];
        double nrm = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI));
        double amp = nrm * orc_wigner_d(l, m, 2, iota), damp = nrm * orc_wigner_d_deriv(l, m, 2, iota);
        y[2 * a] = amp * cos(m * phi);
        y[2 * a + 1] = amp * sin(m * phi);
        dy[2 * a] = damp * cos(m * phi);
        dy[2 * a + 1] = damp * sin(m * phi);
    }
    /* coefficients */
    double *c = (double *)malloc(sizeof(double) * 2 * K * M);
    for (int k = 0; k < K; k++)
        for (int a = 0; a < M; a++) {
            c[2 * (k * M + a)] = sD * (F[2 * k] * y[2 * a] - F[2 * k + 1] * y[2 * a + 1]);
            c[2 * (k * M + a) + 1] = sD * (F[2 * k] * y[2 * a + 1] + F[2 * k + 1] * y[2 * a]);
        }
    /* forward: lnL(j) and softmax weights */
    double *lnL = (double *)malloc(sizeof(double) * Nt);
    double A = quadratic(P, c);
    int status = ORC_OK;
    for (int j = 0; j < Nt; j++) {
        double data = 0.0;
        for (int k = 0; k < K; k++) {
            double x = (tc + ((double)j - 0.5 * Nt) / P->fs + dt[k] - P->t_start) * P->fs;
            double fl = floor(x), w = x - fl;
            if (fl < 0.0 || fl + 1.0 > (double)(T - 1)) { status = ORC_E_RANGE; continue; }
            long i = (long)fl;
            for (int a = 0; a < M; a++) {
                const double *q = P->Q + 2 * (((size_t)k * M + a) * T);
                double qr = (1.0 - w) * q[2 * i] + w * q[2 * (i + 1)];
                double qi = (1.0 - w) * q[2 * i + 1] + w * q[2 * (i + 1) + 1];
                data += c[2 * (k * M + a)] * qr + c[2 * (k * M + a) + 1] * qi;
            }
        }
        lnL[j] = data - A;
    }
    double mx = lnL[0];
    for (int j = 1; j < Nt; j++) if (lnL[j] > mx) mx = lnL[j];
    double ssum = 0.0;
    for (int j = 0; j < Nt; j++) ssum += exp(lnL[j] - mx);
    if (lnL_t_out) *lnL_t_out = mx + log(ssum) - log((double)Nt);
    /* backward through the window: E_ka = sum_j pi_j Qhat_ka(j), slope S_k, gQ */
    double *E = (double *)calloc(2 * K * M, sizeof(double)), *S = (double *)calloc(K, sizeof(double));
    for (int j = 0; j < Nt; j++) {
        double pj = exp(lnL[j] - mx) / ssum;
        for (int k = 0; k < K; k++) {
            double x = (tc + ((double)j - 0.5 * Nt) / P->fs + dt[k] - P->t_start) * P->fs;
            double fl = floor(x), w = x - fl;
            if (fl < 0.0 || fl + 1.0 > (double)(T - 1)) continue;
            long i = (long)fl;
            for (int a = 0; a < M; a++) {
                const double *q = P->Q + 2 * (((size_t)k * M + a) * T);
                double cr = c[2 * (k * M + a)], ci = c[2 * (k * M + a) + 1];
                E[2 * (k * M + a)] += pj * ((1.0 - w) * q[2 * i] + w * q[2 * (i + 1)]);
                E[2 * (k * M + a) + 1] += pj * ((1.0 - w) * q[2 * i + 1] + w * q[2 * (i + 1) + 1]);
                S[k] += pj * (cr * (q[2 * (i + 1)] - q[2 * i]) + ci * (q[2 * (i + 1) + 1] - q[2 * i + 1]));
                if (gQ) {
                    double *gq = gQ + 2 * (((size_t)k * M + a) * T);
                    gq[2 * i] += g * pj * (1.0 - w) * cr;
                    gq[2 * i + 1] += g * pj * (1.0 - w) * ci;
                    gq[2 * (i + 1)] += g * pj * w * cr;
                    gq[2 * (i + 1) + 1] += g * pj * w * ci;
                }
            }
        }
    }
    /* quadratic term: dA/dc (entries of U, V as given, no symmetry assumed) and gU, gV */
    double *gc = (double *)malloc(sizeof(double) * 2 * K * M);
    for (int k = 0; k < K; k++) {
        const double *Uk = P->U + 2 * (size_t)k * M * M, *Vk = P->V + 2 * (size_t)k * M * M;
        const double *ck = c + 2 * k * M;
        for (int a = 0; a < M; a++) {
            /* dA/dc_r,a and dA/dc_i,a */
            double dr = 0.0, di = 0.0;
            for (int b = 0; b < M; b++) {
                double ur = Uk[2 * (a * M + b)], ui = Uk[2 * (a * M + b) + 1];   /* U_ab */
                double uTr = Uk[2 * (b * M + a)], uTi = Uk[2 * (b * M + a) + 1]; /* U_ba */
                double vr = Vk[2 * (a * M + b)], vi = Vk[2 * (a * M + b) + 1];
                double vTr = Vk[2 * (b * M + a)], vTi = Vk[2 * (b * M + a) + 1];
                double cbr = ck[2 * b], cbi = ck[2 * b + 1];
                /* (U c)_a = sum_b U_ab c_b; (c^H U)_a = sum_b conj(c_b) U_ba */
                double Ucr = ur * cbr - ui * cbi, Uci = ur * cbi + ui * cbr;
                double cUr = cbr * uTr + cbi * uTi, cUi = cbr * uTi - cbi * uTr;
                double Vcr = vr * cbr - vi * cbi, Vci = vr * cbi + vi * cbr;
                double cVr = cbr * vTr - cbi * vTi, cVi = cbr * vTi + cbi * vTr;
                /* d/dc_r of conj(c_a)(Uc)_a + (c^H U)_a c_a = (Uc)_a + (c^H U)_a ; d/dc_i: -i(Uc)_a + i (c^H U)_a */
                dr += Ucr + cUr + Vcr + cVr;
                di += (Uci - cUi) + (-(Vci) - cVi);
            }
            gc[2 * (k * M + a)] = E[2 * (k * M + a)] - 0.25 * dr;
            gc[2 * (k * M + a) + 1] = E[2 * (k * M + a) + 1] - 0.25 * di;
            if (gU || gV) {
                for (int b = 0; b < M; b++) {
                    double car = ck[2 * a], cai = ck[2 * a + 1], cbr = ck[2 * b], cbi = ck[2 * b + 1];
                    double pr = car * cbr + cai * cbi, pim = car * cbi - cai * cbr; /* conj(c_a) c_b */
                    double qr = car * cbr - cai * cbi, qim = car * cbi + cai * cbr; /* c_a c_b */
                    if (gU) {
                        gU[2 * ((size_t)(k * M + a) * M + b)] += g * (-0.25 * pr);
                        gU[2 * ((size_t)(k * M + a) * M + b) + 1] += g * (0.25 * pim);
                    }
                    if (gV) {
                        gV[2 * ((size_t)(k * M + a) * M + b)] += g * (-0.25 * qr);
                        gV[2 * ((size_t)(k * M + a) * M + b) + 1] += g * (0.25 * qim);
                    }
                }
            }
        }
    }
    /* chain rule to theta */
    double gth[7] = {0, 0, 0, 0, 0, 0, 0};
    double gs = 0.0;
    for (int k = 0; k < K; k++) {
        double gFr = 0.0, gFi = 0.0;
        for (int a = 0; a < M; a++) {
            double gcr = gc[2 * (k * M + a)], gci = gc[2 * (k * M + a) + 1];
            double yr = y[2 * a], yi = y[2 * a + 1];
            /* c = sD F y:  dc/dFr = sD y, dc/dFi = i sD y */
            gFr += sD * (gcr * yr + gci * yi);
            gFi += sD * (-gcr * yi + gci * yr);
            gs += gcr * c[2 * (k * M + a)] + gci * c[2 * (k * M + a) + 1];
        }
        for (int p = 0; p < 3; p++) gth[p] += gFr * dF[(k * 3 + p) * 2] + gFi * dF[(k * 3 + p) * 2 + 1];
        /* window position x = (tc + dt_k ...) fs */
        gth[6] += S[k] * P->fs;
        gth[0] += S[k] * P->fs * ddt[2 * k];
        gth[1] += S[k] * P->fs * ddt[2 * k + 1];
    }
    gth[5] = -gs / dist; /* c prop. to 1/D */
    for (int a = 0; a < M; a++) {
        int m = P->lm[2 * a + 1];
        double gyr = 0.0, gyi = 0.0;
        for (int k = 0; k < K; k++) {
            double gcr = gc[2 * (k * M + a)], gci = gc[2 * (k * M + a) + 1];
            double fr = sD * F[2 * k], fi = sD * F[2 * k + 1];
            gyr += gcr * fr + gci * fi;
            gyi += -gcr * fi + gci * fr;
        }
        gth[3] += gyr * dy[2 * a] + gyi * dy[2 * a + 1];
        gth[4] += gyr * (-m * y[2 * a + 1]) + gyi * (m * y[2 * a]);
    }
    for (int d = 0; d < 7; d++) g_th[d] += g * gth[d];
    free(F); free(dF); free(dt); free(ddt); free(y); free(dy); free(c); free(lnL); free(E); free(S); free(gc);
    return status;
}

/* ---------------------------------------------------------------- distance marginalisation (R22) */

/*
 * ln F(a, b) = ln int_{D_min}^{D_max} p(D) exp(a x - b x^2) dD,  x = D_ref / D,
 * p(D) = 3 D^2 / (D_max^3 - D_min^3): the distance integral of the likelihood at fixed other
 * parameters, with a the data term and b the quadratic term at D = D_ref (App. "Distance
 * marginalization" names the technique; the integral is written out here).  Composite
 * 32-point Gauss-Legendre in x: 64 equal panels plus panels of geometrically growing width around
 * the exponent's maximum (edges at x* +- l 2^m, l the peak's width or decay length), so that a
 * narrow peak is resolved however large b is; the exponent is shifted by its maximum first.
 */
static void gl32(double *x, double *w)
{
    /* nodes and weights of the 32-point Gauss-Legendre rule on [-1, 1] by Newton on P_32 */
    const int n = 32;
    for (int i = 0; i < n; i++) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; j++) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-15) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

static int cmp_double(const void *p, const void *q)
{
    double a = *(const double *)p, b = *(const double *)q;
    return (a > b) - (a < b);
}

double orc_dmarg_lnF(double a, double b, double d_min, double d_max, double d_ref)
{
    static double gx[32], gw[32];
    static int ready = 0;
    if (!ready) {
        gl32(gx, gw);
        ready = 1;
    }
    /* in x = d_ref / D the prior is C x^-4 dx on [xlo, xhi] and the exponent a x - b x^2 */
    const double xlo = d_ref / d_max, xhi = d_ref / d_min;
    const double C = 3.0 * d_ref * d_ref * d_ref / (d_max * d_max * d_max - d_min * d_min * d_min);
    double xs = b > 0.0 ? a / (2.0 * b) : (a > 0.0 ? xhi : xlo);
    if (xs < xlo) xs = xlo;
    if (xs > xhi) xs = xhi;
    const double shift = a * xs - b * xs * xs; /* the exponent's maximum on the range */
    /* its scale there: 1/sqrt(2b) (peak) or 1/|slope| (decay from an end) */
    const double slope = fabs(a - 2.0 * b * xs);
    double ell = b > 0.0 ? 1.0 / sqrt(2.0 * b) : INFINITY;
    if (slope > 0.0 && 1.0 / slope < ell) ell = 1.0 / slope;
    /* panel edges: 64 equal panels, plus xs +- ell 2^m (m = -3 .. 60), so that the panels next to
     * the peak are a fraction of its width and grow geometrically away from it */
    double e[64 + 1 + 2 * 64 + 1];
    int ne = 0;
    for (int p = 0; p <= 64; p++) e[ne++] = xlo + (xhi - xlo) * p / 64.0;
    e[ne++] = xs;
    for (int m = -3; m <= 60; m++) {
        double d = ell * ldexp(1.0, m);
        if (xs - d > xlo) e[ne++] = xs - d;
        if (xs + d < xhi) e[ne++] = xs + d;
    }
    qsort(e, ne, sizeof(double), cmp_double);
    double s = 0.0;
    for (int p = 0; p + 1 < ne; p++) {
        double lo = e[p], hi = e[p + 1];
        if (!(hi > lo)) continue;
        double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo), t = 0.0;
        for (int i = 0; i < 32; i++) {
            double x = c + h * gx[i];
            t += gw[i] * C / (x * x * x * x) * exp(a * x - b * x * x - shift);
        }
        s += h * t;
    }
    return shift + log(s);
}

/* Distance-marginalised, time-marginalised lnL of N samples: LSE_j ln F(data_j, A) - ln N_t,
 * data_j and A evaluated at D = D_ref (the samples' own D is ignored). */
int orc_lnL_dmarg(const orc_point *P, const double *samples, long N, double d_min, double d_max, double *out)
{
    int status = ORC_OK, Nt = P->n_window;
    double dummy = orc_dmarg_lnF(0.0, 0.0, d_min, d_max, P->d_ref); /* fills the rule before the threads start */
    (void)dummy;
#pragma omp parallel
    {
    double *lnL = (double *)malloc(sizeof(double) * Nt), *data = (double *)malloc(sizeof(double) * Nt);
#pragma omp for schedule(dynamic, 4)
    for (long n = 0; n < N; n++) {
        double th[7], A = 0.0;
        for (int d = 0; d < 7; d++) th[d] = samples[(size_t)d * N + n];
        th[5] = P->d_ref;
        int st = orc_lnL_grid(P, th, lnL, data, &A);
        if (st != ORC_OK) {
#pragma omp atomic write
            status = st;
        }
        double m = -INFINITY;
        for (int j = 0; j < Nt; j++) {
            lnL[j] = orc_dmarg_lnF(data[j], A, d_min, d_max, P->d_ref);
            if (lnL[j] > m) m = lnL[j];
        }
        double s = 0.0;
        for (int j = 0; j < Nt; j++) s += exp(lnL[j] - m);
        out[n] = m + log(s) - log((double)Nt);
    }
    free(lnL);
    free(data);
    }
    return status;
}
