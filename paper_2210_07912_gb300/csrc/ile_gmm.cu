// ile_gmm.cu -- Gaussian-mixture adaptation of the sampling prior (Sec. "Adaptive sampling with
// gaussian mixture models"; App. "Gaussian mixture model implementation"), separable form: each
// adaptive dimension in the mixture mask has its own one-dimensional mixture of normals truncated
// to the dimension's range.
//
// Per iteration and mixture dimension:
//   em_iters x { gmm_em_partial: one pass over the iteration's samples; every thread accumulates,
//                for each component c, S0 = sum q, S1 = sum q (u - m_c), S2 = sum q (u - m_c)^2
//                with q = w_n r_nc (responsibilities from the untruncated normals, computed as a
//                log-sum-exp in FP32; sums in FP64, centred on the component's current mean m_c so
//                that the variance does not cancel), plus W = sum w_n; one row of partial sums per
//                block (fixed grid, so the result does not depend on scheduling);
//              gmm_em_finalize: sums the rows in block order and applies the M-step }
//   the last finalize also merges the batch mixture into the current one (component matching by
//   the least total Mahalanobis distance over all permutations, searched by one warp) and
//   rebuilds the FP32 sampler table.
// The sample weights are w_n = exp(ln w_n - max ln w) with ln w_n = lnL_t + ln p - ln p_s, the
// same weights the histogram sampler uses.
#include <math.h>
#include <stdint.h>

#include "ile_internal.cuh"

namespace {

constexpr int EM_BLOCKS = 304;  // 2 x 152 SMs, grid-stride
constexpr int EM_THREADS = 256;
constexpr int NSTAT = 3 * ILE_GMM_MAX + 1;  // S0, S1, S2 per component, W

struct GmmDims {
    int n;
    int d[ILE_NDIM];
};

GmmDims dims_of(unsigned mask) {
    GmmDims g{};
    for (int d = 0; d < ILE_NDIM; d++)
        if (mask & (1u << d)) g.d[g.n++] = d;
    return g;
}

// FP32 sampler form of one mixture; the integer weight table uses explicit round-to-nearest
// operations so that it is the same on every implementation of the definition.
__device__ void build_table(const IleGmm &g, IleGmmTab &t) {
    const int C = g.C;
    double tot = 0.0;
    for (int c = 0; c < C; c++) tot = __dadd_rn(tot, g.w[c]);
    double acc = 0.0;
    t.cw[0] = 0;
    for (int c = 0; c < C; c++) {
        acc = __dadd_rn(acc, __ddiv_rn(g.w[c], tot));
        if (c + 1 < C) {
            double v = floor(__dmul_rn(acc, 4294967296.0));
            if (v > 4294967296.0) v = 4294967296.0;
            t.cw[c + 1] = (uint64_t)v;
        }
    }
    t.cw[C] = (uint64_t)1 << 32;
    for (int c = 1; c <= C; c++)
        if (t.cw[c] < t.cw[c - 1]) t.cw[c] = t.cw[c - 1];
    const double s2pi = sqrt(2.0 * 3.14159265358979323846);
    for (int c = 0; c < ILE_GMM_MAX; c++) {
        if (c < C) {
            const double zl = (g.lo - g.mu[c]) / g.sigma[c], zh = (g.hi - g.mu[c]) / g.sigma[c];
            const double p1 = normcdf(zl), Z = normcdf(zh) - p1;
            t.mu[c] = (float)g.mu[c];
            t.sig[c] = (float)g.sigma[c];
            t.p1[c] = (float)p1;
            t.q2[c] = (float)normcdf(-zh);
            t.dm[c] = (float)Z;
            t.coef[c] = (float)(log(g.w[c] / tot) - log(s2pi * g.sigma[c] * Z));
        } else {
            t.mu[c] = t.sig[c] = t.p1[c] = t.q2[c] = t.dm[c] = 0.f;
            t.coef[c] = -INFINITY;
        }
    }
    t.C = C;
}

__global__ void gmm_table_kernel(GmmDims dims, const IleGmm *__restrict__ cur, IleGmmTab *__restrict__ tab) {
    const int i = threadIdx.x;
    if (i < dims.n) build_table(cur[dims.d[i]], tab[dims.d[i]]);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// grid (EM_BLOCKS, n mixture dimensions); model: the mixture the E-step uses (cur or bat)
__global__ void __launch_bounds__(EM_THREADS) gmm_em_partial_kernel(GmmDims dims, const IleGmm *__restrict__ model,
                                                                    const float *__restrict__ u_all,
                                                                    const double *__restrict__ lnL,
                                                                    const double *__restrict__ lnwp,
                                                                    const double *__restrict__ iter_res, int64_t N,
                                                                    double *__restrict__ part) {
    const int slot = blockIdx.y, d = dims.d[slot];
    __shared__ float mu_s[ILE_GMM_MAX], isg_s[ILE_GMM_MAX], lw_s[ILE_GMM_MAX];
    __shared__ double red[EM_THREADS / 32][NSTAT];
    const int C = model[d].C;
    if (threadIdx.x < ILE_GMM_MAX) {
        const int c = threadIdx.x;
        const IleGmm &g = model[d];
        mu_s[c] = c < C ? (float)g.mu[c] : 0.f;
        isg_s[c] = c < C ? (float)(1.0 / g.sigma[c]) : 0.f;
        lw_s[c] = c < C ? (float)log(g.w[c] / g.sigma[c]) : -INFINITY;
    }
    __syncthreads();
    double acc[NSTAT];
#pragma unroll
    for (int k = 0; k < NSTAT; k++) acc[k] = 0.0;
    const double m = iter_res[4];
    const float *u = u_all + (int64_t)slot * N;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const double w = exp(lnL[n] + lnwp[n] - m);
        const float x = u[n];
        float l[ILE_GMM_MAX], lm = -INFINITY;
#pragma unroll
        for (int c = 0; c < ILE_GMM_MAX; c++) {
            const float z = (x - mu_s[c]) * isg_s[c];
            l[c] = c < C ? lw_s[c] - 0.5f * z * z : -INFINITY;
            lm = fmaxf(lm, l[c]);
        }
        float tot = 0.f;
#pragma unroll
        for (int c = 0; c < ILE_GMM_MAX; c++) {
            l[c] = c < C ? __expf(l[c] - lm) : 0.f;
            tot += l[c];
        }
        const double wt = w / (double)tot;
#pragma unroll
        for (int c = 0; c < ILE_GMM_MAX; c++) {
            if (c < C) {
                const double q = wt * (double)l[c], dx = (double)(x - mu_s[c]);
                acc[3 * c] += q;
                acc[3 * c + 1] += q * dx;
                acc[3 * c + 2] += q * dx * dx;
            }
        }
        acc[NSTAT - 1] += w;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NSTAT; k++) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NSTAT) {
        double s = 0.0;
        for (int w = 0; w < EM_THREADS / 32; w++) s += red[w][threadIdx.x];
        part[((int64_t)slot * gridDim.x + blockIdx.x) * NSTAT + threadIdx.x] = s;
    }
}

__device__ __forceinline__ int factorial(int n) {
    int f = 1;
    for (int i = 2; i <= n; i++) f *= i;
    return f;
}

// k-th permutation of 0..C-1 in lexicographic order.
__device__ void unrank(int k, int C, int perm[ILE_GMM_MAX]) {
    int avail[ILE_GMM_MAX];
    for (int i = 0; i < C; i++) avail[i] = i;
    int navail = C;
    for (int a = 0; a < C; a++) {
        const int f = factorial(C - 1 - a);
        const int idx = k / f;
        k -= idx * f;
        perm[a] = avail[idx];
        for (int i = idx; i + 1 < navail; i++) avail[i] = avail[i + 1];
        navail--;
    }
}

// One warp per mixture dimension: M-step from the block sums; on the last EM step also the merge
// into cur (N = n_samples) and the new sampler table.
__global__ void __launch_bounds__(32) gmm_em_finalize_kernel(GmmDims dims, const double *__restrict__ part,
                                                             int nblk, const IleGmm *__restrict__ in,
                                                             IleGmm *__restrict__ bat, IleGmm *__restrict__ cur,
                                                             IleGmmTab *__restrict__ tab, int last, int64_t N) {
    const int slot = blockIdx.x, d = dims.d[slot], t = threadIdx.x;
    __shared__ double S[NSTAT];
    __shared__ IleGmm gb;
    __shared__ double cost[ILE_GMM_MAX][ILE_GMM_MAX];
    if (t < NSTAT) {
        double s = 0.0;
        for (int b = 0; b < nblk; b++) s += part[((int64_t)slot * nblk + b) * NSTAT + t];
        S[t] = s;
    }
    __syncwarp();
    if (t == 0) {
        IleGmm g = in[d];
        const double W = S[NSTAT - 1];
        if (W > 0.0) {
            const double smin = (g.hi - g.lo) * 1e-3;
            double wsum = 0.0;
            for (int c = 0; c < g.C; c++) {
                if (S[3 * c] > 1e-12 * W) {
                    const double ref = (double)(float)g.mu[c];  // the centre of the partial sums
                    const double m1 = S[3 * c + 1] / S[3 * c];
                    const double var = S[3 * c + 2] / S[3 * c] - m1 * m1;
                    g.mu[c] = fmin(fmax(ref + m1, g.lo), g.hi);
                    g.sigma[c] = sqrt(fmax(var, smin * smin));
                    g.w[c] = S[3 * c] / W;
                } else {
                    g.w[c] = 1e-3;
                }
                wsum += g.w[c];
            }
            for (int c = 0; c < g.C; c++) g.w[c] /= wsum;
        }
        gb = g;
        if (!last) bat[d] = g;
    }
    __syncwarp();
    if (!last) return;
    // merge: the first permutation (lexicographic) of least total Mahalanobis distance
    const IleGmm &cu = cur[d];
    const int C = cu.C;
    if (t < C * C) {
        const int a = t / C, j = t % C;
        cost[a][j] = fabs(cu.mu[j] - gb.mu[a]) / gb.sigma[a] + fabs(gb.mu[a] - cu.mu[j]) / cu.sigma[j];
    }
    __syncwarp();
    const int nperm = factorial(C);
    double best = INFINITY;
    int bestk = nperm;
    for (int k = t; k < nperm; k += 32) {
        int perm[ILE_GMM_MAX];
        unrank(k, C, perm);
        double c = 0.0;
        for (int a = 0; a < C; a++) c += cost[a][perm[a]];
        if (c < best) {
            best = c;
            bestk = k;
        }
    }
    for (int o = 16; o; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int ok = __shfl_xor_sync(0xffffffffu, bestk, o);
        if (ob < best || (ob == best && ok < bestk)) {
            best = ob;
            bestk = ok;
        }
    }
    if (t == 0) {
        int perm[ILE_GMM_MAX];
        unrank(bestk < nperm ? bestk : 0, C, perm);
        IleGmm out = cu;
        const double Nold = cu.n, M = (double)N;
        for (int a = 0; a < C; a++) {
            const int j = perm[a];
            const double A = Nold * cu.w[j], B = M * gb.w[a];
            const double mu = (A * cu.mu[j] + B * gb.mu[a]) / (A + B);
            const double var = (A * cu.sigma[j] * cu.sigma[j] + B * gb.sigma[a] * gb.sigma[a]) / (A + B) +
                               (A * cu.mu[j] * cu.mu[j] + B * gb.mu[a] * gb.mu[a]) / (A + B) - mu * mu;
            out.mu[a] = mu;
            out.sigma[a] = sqrt(fmax(var, 0.0));
            out.w[a] = (A + B) / (Nold + M);
        }
        out.n = Nold + M;
        cur[d] = out;
        build_table(out, tab[d]);
    }
}

// ------------------------------------------------------------------ the correlated sky pair
//
// Component c of the pair is a bivariate normal N(mu_c, cov_c) truncated to the rectangle R of
// sampling variables 0 and 1.  Sampling draws whitened standard normals truncated to the box that
// holds L_c^-1 (R - mu_c) and rejects points outside R (ile_adapt.cu), so the accepted density of
// the component is N / Z_c on R with Z_c its mass there; Z_c is the integral over the first
// standardised coordinate u of phi(u) [Phi((b - rho u) / s) - Phi((a - rho u) / s)] (the
// conditional law of the second), by composite Gauss-Legendre quadrature.

constexpr int NSTAT2 = 6 * ILE_GMM_MAX + 1;  // S0, S1x, S1y, Sxx, Sxy, Syy per component, W
constexpr int GL_N = 16, GL_PANELS = 32;     // Z_c: 32 panels x 16-point Gauss-Legendre

struct GlRule {
    double x[GL_N], w[GL_N];  // nodes and weights on [-1, 1]
};

// Gauss-Legendre nodes and weights (Newton iteration on the Legendre polynomial), once per process.
GlRule gl_rule() {
    static GlRule r = [] {
        GlRule g{};
        for (int i = 0; i < GL_N; i++) {
            double x = cos(3.14159265358979323846 * (i + 0.75) / (GL_N + 0.5)), dp = 1.0;
            for (int it = 0; it < 100; it++) {
                double p0 = 1.0, p1 = x;
                for (int k = 2; k <= GL_N; k++) {
                    const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = GL_N * (x * p1 - p0) / (x * x - 1.0);
                const double dx = p1 / dp;
                x -= dx;
                if (fabs(dx) < 1e-16) break;
            }
            g.x[i] = x;
            g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
        }
        return g;
    }();
    return r;
}

// Mass of R under N(mu, cov) (see above); the first coordinate's range is cut to [-12, 12] sigma.
__device__ double bvn_rect(const GlRule &gl, const double mu[2], const double cov[3], const double lo[2],
                           const double hi[2]) {
    const double s0 = sqrt(cov[0]), s1 = sqrt(cov[2]);
    const double rho = cov[1] / (s0 * s1), sr = sqrt(1.0 - rho * rho);
    const double a0 = fmax((lo[0] - mu[0]) / s0, -12.0), b0 = fmin((hi[0] - mu[0]) / s0, 12.0);
    const double a1 = (lo[1] - mu[1]) / s1, b1 = (hi[1] - mu[1]) / s1;
    if (!(b0 > a0)) return 0.0;
    const double h = (b0 - a0) / GL_PANELS;
    double sum = 0.0;
    for (int p = 0; p < GL_PANELS; p++) {
        const double mid = a0 + (p + 0.5) * h;
        for (int i = 0; i < GL_N; i++) {
            const double u = mid + 0.5 * h * gl.x[i];
            const double f = exp(-0.5 * u * u) * (normcdf((b1 - rho * u) / sr) - normcdf((a1 - rho * u) / sr));
            sum += gl.w[i] * f;
        }
    }
    return sum * 0.5 * h / sqrt(2.0 * 3.14159265358979323846);
}

// FP32 sampler form of the pair (IleGmm2Tab); the integer weight table as in build_table.
__device__ void build_table2(const GlRule &gl, const IleGmm2 &g, IleGmm2Tab &t) {
    const int C = g.C;
    double tot = 0.0;
    for (int c = 0; c < C; c++) tot = __dadd_rn(tot, g.w[c]);
    double acc = 0.0;
    t.cw[0] = 0;
    for (int c = 0; c < C; c++) {
        acc = __dadd_rn(acc, __ddiv_rn(g.w[c], tot));
        if (c + 1 < C) {
            double v = floor(__dmul_rn(acc, 4294967296.0));
            if (v > 4294967296.0) v = 4294967296.0;
            t.cw[c + 1] = (uint64_t)v;
        }
    }
    t.cw[C] = (uint64_t)1 << 32;
    for (int c = 1; c <= C; c++)
        if (t.cw[c] < t.cw[c - 1]) t.cw[c] = t.cw[c - 1];
    for (int c = 0; c < ILE_GMM_MAX; c++) {
        if (c >= C) {
            t.coef[c] = -INFINITY;
            continue;
        }
        const double *S = g.cov[c];
        const double l0 = sqrt(S[0]), l1 = S[1] / l0, l2 = sqrt(S[2] - l1 * l1);
        double blo[2] = {INFINITY, INFINITY}, bhi[2] = {-INFINITY, -INFINITY};
        for (int k = 0; k < 4; k++) {
            const double x0 = (k & 1) ? g.hi[0] : g.lo[0], x1 = (k & 2) ? g.hi[1] : g.lo[1];
            const double y0 = (x0 - g.mu[c][0]) / l0, y1 = (x1 - g.mu[c][1] - l1 * y0) / l2;
            blo[0] = fmin(blo[0], y0);
            bhi[0] = fmax(bhi[0], y0);
            blo[1] = fmin(blo[1], y1);
            bhi[1] = fmax(bhi[1], y1);
        }
        const double det = S[0] * S[2] - S[1] * S[1];
        const double Z = bvn_rect(gl, g.mu[c], S, g.lo, g.hi);
        for (int j = 0; j < 2; j++) {
            t.mu[c][j] = (float)g.mu[c][j];
            t.p1[c][j] = (float)normcdf(blo[j]);
            t.q2[c][j] = (float)normcdf(-bhi[j]);
            t.dm[c][j] = (float)(normcdf(bhi[j]) - normcdf(blo[j]));
        }
        t.L[c][0] = (float)l0;
        t.L[c][1] = (float)l1;
        t.L[c][2] = (float)l2;
        t.icov[c][0] = (float)(S[2] / det);
        t.icov[c][1] = (float)(-S[1] / det);
        t.icov[c][2] = (float)(S[0] / det);
        t.coef[c] = (float)(log(g.w[c] / tot) - log(2.0 * 3.14159265358979323846 * sqrt(det) * Z));
    }
    t.C = C;
}

__global__ void gmm2_table_kernel(GlRule gl, const IleGmm2 *__restrict__ cur, IleGmm2Tab *__restrict__ tab) {
    if (threadIdx.x == 0) build_table2(gl, *cur, *tab);
}

// E-step partial sums of the pair over a grid-stride share of the samples; the sums are centred
// on each component's current mean (rounded to FP32, the value the responsibilities use).
__global__ void __launch_bounds__(EM_THREADS) gmm2_em_partial_kernel(const IleGmm2 *__restrict__ model,
                                                                     const float *__restrict__ u_pair,
                                                                     const double *__restrict__ lnL,
                                                                     const double *__restrict__ lnwp,
                                                                     const double *__restrict__ iter_res, int64_t N,
                                                                     double *__restrict__ part) {
    __shared__ float mu_s[ILE_GMM_MAX][2], ic_s[ILE_GMM_MAX][3], lw_s[ILE_GMM_MAX];
    __shared__ double red[EM_THREADS / 32][NSTAT2];
    const int C = model->C;
    if (threadIdx.x < ILE_GMM_MAX) {
        const int c = threadIdx.x;
        const IleGmm2 &g = *model;
        if (c < C) {
            const double *S = g.cov[c];
            const double det = S[0] * S[2] - S[1] * S[1];
            mu_s[c][0] = (float)g.mu[c][0];
            mu_s[c][1] = (float)g.mu[c][1];
            ic_s[c][0] = (float)(S[2] / det);
            ic_s[c][1] = (float)(-S[1] / det);
            ic_s[c][2] = (float)(S[0] / det);
            lw_s[c] = (float)(log(g.w[c]) - 0.5 * log(det));
        } else {
            mu_s[c][0] = mu_s[c][1] = ic_s[c][0] = ic_s[c][1] = ic_s[c][2] = 0.f;
            lw_s[c] = -INFINITY;
        }
    }
    __syncthreads();
    double acc[NSTAT2];
#pragma unroll
    for (int k = 0; k < NSTAT2; k++) acc[k] = 0.0;
    const double m = iter_res[4];
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const double w = exp(lnL[n] + lnwp[n] - m);
        const float x0 = u_pair[n], x1 = u_pair[N + n];
        float l[ILE_GMM_MAX], lm = -INFINITY;
#pragma unroll
        for (int c = 0; c < ILE_GMM_MAX; c++) {
            const float d0 = x0 - mu_s[c][0], d1 = x1 - mu_s[c][1];
            const float q = ic_s[c][0] * d0 * d0 + 2.f * ic_s[c][1] * d0 * d1 + ic_s[c][2] * d1 * d1;
            l[c] = c < C ? lw_s[c] - 0.5f * q : -INFINITY;
            lm = fmaxf(lm, l[c]);
        }
        float tot = 0.f;
#pragma unroll
        for (int c = 0; c < ILE_GMM_MAX; c++) {
            l[c] = c < C ? __expf(l[c] - lm) : 0.f;
            tot += l[c];
        }
        const double wt = w / (double)tot;
#pragma unroll
        for (int c = 0; c < ILE_GMM_MAX; c++) {
            if (c < C) {
                const double q = wt * (double)l[c], d0 = (double)(x0 - mu_s[c][0]), d1 = (double)(x1 - mu_s[c][1]);
                acc[6 * c] += q;
                acc[6 * c + 1] += q * d0;
                acc[6 * c + 2] += q * d1;
                acc[6 * c + 3] += q * d0 * d0;
                acc[6 * c + 4] += q * d0 * d1;
                acc[6 * c + 5] += q * d1 * d1;
            }
        }
        acc[NSTAT2 - 1] += w;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NSTAT2; k++) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NSTAT2) {
        double s = 0.0;
        for (int w = 0; w < EM_THREADS / 32; w++) s += red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * NSTAT2 + threadIdx.x] = s;
    }
}

// sigma_j >= 1e-3 of the range, |rho| <= 0.9, the mean inside the rectangle
__device__ void pair_floor(IleGmm2 &g, int c) {
    double *S = g.cov[c];
    for (int j = 0; j < 2; j++) {
        const double smin = 1e-3 * (g.hi[j] - g.lo[j]);
        S[2 * j] = fmax(S[2 * j], smin * smin);
        g.mu[c][j] = fmin(fmax(g.mu[c][j], g.lo[j]), g.hi[j]);
    }
    const double lim = 0.9 * sqrt(S[0] * S[2]);
    S[1] = fmin(fmax(S[1], -lim), lim);
}

__device__ double mahalanobis2(double d0, double d1, const double S[3]) {
    const double det = S[0] * S[2] - S[1] * S[1];
    return sqrt((S[2] * d0 * d0 - 2.0 * S[1] * d0 * d1 + S[0] * d1 * d1) / det);
}

// One warp: M-step from the block sums; on the last EM step the merge into cur (the permutation of
// least summed two-sided Mahalanobis distance, first in lexicographic order; N = n_samples) and
// the new sampler table.
__global__ void __launch_bounds__(32) gmm2_em_finalize_kernel(GlRule gl, const double *__restrict__ part, int nblk,
                                                              const IleGmm2 *__restrict__ in,
                                                              IleGmm2 *__restrict__ bat, IleGmm2 *__restrict__ cur,
                                                              IleGmm2Tab *__restrict__ tab, int last, int64_t N) {
    const int t = threadIdx.x;
    __shared__ double S[NSTAT2];
    __shared__ IleGmm2 gb;
    __shared__ double cost[ILE_GMM_MAX][ILE_GMM_MAX];
    for (int k = t; k < NSTAT2; k += 32) {
        double s = 0.0;
        for (int b = 0; b < nblk; b++) s += part[(int64_t)b * NSTAT2 + k];
        S[k] = s;
    }
    __syncwarp();
    if (t == 0) {
        IleGmm2 g = *in;
        const double W = S[NSTAT2 - 1];
        if (W > 0.0) {
            double wsum = 0.0;
            for (int c = 0; c < g.C; c++) {
                const double *s6 = S + 6 * c;
                if (s6[0] > 1e-12 * W) {
                    const double r0 = (double)(float)g.mu[c][0], r1 = (double)(float)g.mu[c][1];
                    const double m0 = s6[1] / s6[0], m1 = s6[2] / s6[0];
                    g.mu[c][0] = r0 + m0;
                    g.mu[c][1] = r1 + m1;
                    g.cov[c][0] = s6[3] / s6[0] - m0 * m0;
                    g.cov[c][1] = s6[4] / s6[0] - m0 * m1;
                    g.cov[c][2] = s6[5] / s6[0] - m1 * m1;
                    pair_floor(g, c);
                    g.w[c] = s6[0] / W;
                } else {
                    g.w[c] = 1e-3;
                }
                wsum += g.w[c];
            }
            for (int c = 0; c < g.C; c++) g.w[c] /= wsum;
        }
        gb = g;
        if (!last) *bat = g;
    }
    __syncwarp();
    if (!last) return;
    const IleGmm2 &cu = *cur;
    const int C = cu.C;
    for (int k = t; k < C * C; k += 32) {
        const int a = k / C, j = k % C;
        const double d0 = cu.mu[j][0] - gb.mu[a][0], d1 = cu.mu[j][1] - gb.mu[a][1];
        cost[a][j] = mahalanobis2(d0, d1, gb.cov[a]) + mahalanobis2(d0, d1, cu.cov[j]);
    }
    __syncwarp();
    const int nperm = factorial(C);
    double best = INFINITY;
    int bestk = nperm;
    for (int k = t; k < nperm; k += 32) {
        int perm[ILE_GMM_MAX];
        unrank(k, C, perm);
        double c = 0.0;
        for (int a = 0; a < C; a++) c += cost[a][perm[a]];
        if (c < best) {
            best = c;
            bestk = k;
        }
    }
    for (int o = 16; o; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int ok = __shfl_xor_sync(0xffffffffu, bestk, o);
        if (ob < best || (ob == best && ok < bestk)) {
            best = ob;
            bestk = ok;
        }
    }
    if (t == 0) {
        int perm[ILE_GMM_MAX];
        unrank(bestk < nperm ? bestk : 0, C, perm);
        IleGmm2 out = cu;
        const double Nold = cu.n, M = (double)N;
        for (int a = 0; a < C; a++) {
            const int j = perm[a];
            const double A = Nold * cu.w[j], B = M * gb.w[a];
            const double m0 = (A * cu.mu[j][0] + B * gb.mu[a][0]) / (A + B);
            const double m1 = (A * cu.mu[j][1] + B * gb.mu[a][1]) / (A + B);
            out.mu[a][0] = m0;
            out.mu[a][1] = m1;
            out.cov[a][0] = (A * cu.cov[j][0] + B * gb.cov[a][0]) / (A + B) +
                            (A * cu.mu[j][0] * cu.mu[j][0] + B * gb.mu[a][0] * gb.mu[a][0]) / (A + B) - m0 * m0;
            out.cov[a][1] = (A * cu.cov[j][1] + B * gb.cov[a][1]) / (A + B) +
                            (A * cu.mu[j][0] * cu.mu[j][1] + B * gb.mu[a][0] * gb.mu[a][1]) / (A + B) - m0 * m1;
            out.cov[a][2] = (A * cu.cov[j][2] + B * gb.cov[a][2]) / (A + B) +
                            (A * cu.mu[j][1] * cu.mu[j][1] + B * gb.mu[a][1] * gb.mu[a][1]) / (A + B) - m1 * m1;
            out.w[a] = (A + B) / (Nold + M);
            pair_floor(out, a);
        }
        out.n = Nold + M;
        *cur = out;
        build_table2(gl, out, *tab);
    }
}

}  // namespace

size_t ile_gmm2_part_doubles() { return (size_t)EM_BLOCKS * NSTAT2; }

void ile_gmm2_init(IleGmm2 &g, int C, const double lo[2], const double hi[2]) {
    g = IleGmm2{};
    g.C = C;
    for (int j = 0; j < 2; j++) {
        g.lo[j] = lo[j];
        g.hi[j] = hi[j];
    }
    for (int c = 0; c < C; c++) {
        g.w[c] = 1.0 / C;
        for (int j = 0; j < 2; j++) g.mu[c][j] = lo[j] + (c + 0.5) * (hi[j] - lo[j]) / C;
        g.cov[c][0] = ((hi[0] - lo[0]) / C) * ((hi[0] - lo[0]) / C);
        g.cov[c][1] = 0.0;
        g.cov[c][2] = ((hi[1] - lo[1]) / C) * ((hi[1] - lo[1]) / C);
    }
    g.n = 0.0;
}

cudaError_t ile_launch_gmm2_table(const IleGmm2 *cur, IleGmm2Tab *tab, cudaStream_t st) {
    gmm2_table_kernel<<<1, 32, 0, st>>>(gl_rule(), cur, tab);
    return cudaGetLastError();
}

cudaError_t ile_launch_gmm2_update(const float *u_pair, const double *lnL, const double *lnw_prior,
                                   const double *iter_res, int64_t N, int em_iters, IleGmm2 *cur, IleGmm2 *bat,
                                   IleGmm2Tab *tab, double *part, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const GlRule gl = gl_rule();
    for (int it = 0; it < em_iters; it++) {
        const IleGmm2 *in = it == 0 ? cur : bat;
        gmm2_em_partial_kernel<<<EM_BLOCKS, EM_THREADS, 0, st>>>(in, u_pair, lnL, lnw_prior, iter_res, N, part);
        gmm2_em_finalize_kernel<<<1, 32, 0, st>>>(gl, part, EM_BLOCKS, in, bat, cur, tab, it + 1 == em_iters ? 1 : 0,
                                                  N);
    }
    return cudaGetLastError();
}

size_t ile_gmm_part_doubles() { return (size_t)ILE_NDIM * EM_BLOCKS * NSTAT; }

cudaError_t ile_launch_gmm_table(unsigned mask, const IleGmm *cur, IleGmmTab *tab, cudaStream_t st) {
    const GmmDims dims = dims_of(mask);
    if (dims.n == 0) return cudaSuccess;
    gmm_table_kernel<<<1, 32, 0, st>>>(dims, cur, tab);
    return cudaGetLastError();
}

cudaError_t ile_launch_gmm_update(unsigned mask, const float *u_gmm, const double *lnL, const double *lnw_prior,
                                  const double *iter_res, int64_t N, int em_iters, IleGmm *cur, IleGmm *bat,
                                  IleGmmTab *tab, double *part, cudaStream_t st) {
    const GmmDims dims = dims_of(mask);
    if (dims.n == 0 || N <= 0) return cudaSuccess;
    for (int it = 0; it < em_iters; it++) {
        const IleGmm *in = it == 0 ? cur : bat;
        gmm_em_partial_kernel<<<dim3(EM_BLOCKS, dims.n), EM_THREADS, 0, st>>>(dims, in, u_gmm, lnL, lnw_prior, iter_res,
                                                                              N, part);
        gmm_em_finalize_kernel<<<dims.n, 32, 0, st>>>(dims, part, EM_BLOCKS, in, bat, cur, tab,
                                                      it + 1 == em_iters ? 1 : 0, N);
    }
    return cudaGetLastError();
}
