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

}  // namespace

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
