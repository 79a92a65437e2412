// ile_adapt.cu -- the adaptive-Cartesian Monte Carlo integrator on the device: sample generation
// (S0) and the weighted histograms that adapt the sampling prior (S6), Sec. "GPU-accelerated
// Monte Carlo integration".
//
// The sampling prior is separable, p_s = prod_d p_{s,d}.  Each dimension d has a sampling
// variable u_d on [lo_d, hi_d] (ra, sin dec, psi, cos iota, phi, D, t_c).  A fixed dimension is
// drawn from its prior (uniform, or prop. to D^2 for the distance); an adaptive one from a 100-bin
// piecewise-uniform density given by an integer cumulative table cdf[0..100] (cdf[0] = 0,
// cdf[100] = 2^32): the bin is the largest b with cdf[b] <= a for a 32-bit uniform word a, the
// position inside the bin comes from a second word.  Words: Philox4x32-10 (Salmon et al., SC'11)
// keyed by the seed, counter (sample, iteration, point, block).  Because the bin choice is an
// integer comparison, it is reproduced bit for bit by any implementation of the same definition.
//
// A dimension in the mixture mask is drawn from its truncated Gaussian mixture instead (tables
// built in ile_gmm.cu): component = largest c with cw[c] <= a, u = mu_c + sigma_c Phi^-1(P1_c + v
// Z_c) with v from the second word (evaluated from the nearer tail), ln p_s a log-sum-exp over the
// components; the bins byte holds the component and u is kept for the EM update.
//
// After the likelihood, each adaptive dimension's histogram h_b = sum_{n in b} w_n / sum w
// (w_n = exp(ln w_n - max ln w) <= 1) is accumulated as 2^-40 fixed-point integers (exact and
// independent of the order of the atomics, so a run is reproducible bit for bit); the next table
// is mass_b = (1 - eps) h_b + eps / 100, accumulated left to right in FP64 (explicit
// round-to-nearest operations, no contraction) and cut to cdf[b] = floor(2^32 sum_{b' < b} mass_b').
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>
#include <stdint.h>

#include "ile_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int NB = ILE_NBINS;
constexpr int ND = ILE_NDIM;
constexpr int HIST_THREADS = 256;
constexpr int HIST_CHUNK = 1024;

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t out[4]) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
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

// Known-answer check of the generator: out[i] = Philox4x32-10(counter ck[6i .. 6i+3], key ck[6i+4 .. 6i+5]).
__global__ void philox_kat_kernel(const uint32_t *__restrict__ ck, int64_t n, uint32_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t *c = ck + 6 * i;
    uint32_t w[4];
    philox4x32_10(c[0], c[1], c[2], c[3], c[4], c[5], w);
    for (int q = 0; q < 4; q++) out[4 * i + q] = w[q];
}

// Uniform in (0, 1) from the top 23 bits of a word (exact in FP32).
__device__ __forceinline__ float unit23(uint32_t w) { return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f); }

struct SamplerTables {
    uint32_t cdf[ND][NB + 1];  // low 32 bits; cdf[100] = 2^32 is never compared against
    float lnps[ND][NB];
    IleGmmTab gmm[ND];
    IleGmm2Tab pair;
};

__device__ __forceinline__ void load_tables(SamplerTables &t, const uint64_t *__restrict__ cdf,
                                            const float *__restrict__ lnps_tab, const IleGmmTab *__restrict__ gmm,
                                            unsigned gmm_mask, const IleGmm2Tab *__restrict__ pair = nullptr) {
    if (pair) {
        constexpr int W2 = sizeof(IleGmm2Tab) / 4;
        static_assert(sizeof(IleGmm2Tab) % 4 == 0, "table copied as words");
        const uint32_t *src = reinterpret_cast<const uint32_t *>(pair);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&t.pair);
        for (int i = threadIdx.x; i < W2; i += blockDim.x) dst[i] = src[i];
    }
    for (int i = threadIdx.x; i < ND * (NB + 1); i += blockDim.x) {
        const int d = i / (NB + 1), b = i % (NB + 1);
        t.cdf[d][b] = (uint32_t)cdf[i];
        if (b < NB) t.lnps[d][b] = lnps_tab[d * NB + b];
    }
    if (gmm_mask) {
        constexpr int W = sizeof(IleGmmTab) / 4;
        static_assert(sizeof(IleGmmTab) % 4 == 0, "table copied as words");
        const uint32_t *src = reinterpret_cast<const uint32_t *>(gmm);
        uint32_t *dst = reinterpret_cast<uint32_t *>(t.gmm);
        for (int i = threadIdx.x; i < ND * W; i += blockDim.x) dst[i] = src[i];
    }
}

// One draw from dimension d's truncated mixture: returns u, sets the component and ln p_s.
__device__ __forceinline__ float gmm_draw(const IleGmmTab &g, float lo, float hi, uint32_t a, uint32_t bw, int &comp,
                                          float &lnps) {
    int c = 0;
    for (int j = 1; j < g.C; j++)
        if (g.cw[j] <= (uint64_t)a) c = j;
    // inverse CDF at P = Phi(z_lo) + v Z, taken from the nearer tail so that P never rounds to 1:
    // P <= 1/2: z = Phi^-1(P); otherwise z = -Phi^-1(1 - P), 1 - P = Phi(-z_hi) + (1 - v) Z
    // (both sums of positive terms; 1 - v is exact for the 23-bit v)
    const float v = unit23(bw);
    const float p = g.p1[c] + v * g.dm[c];
    const float z = p <= 0.5f ? normcdfinvf(p) : -normcdfinvf(g.q2[c] + (1.f - v) * g.dm[c]);
    float u = g.mu[c] + g.sig[c] * z;
    u = fminf(fmaxf(u, lo), hi);
    float l[ILE_GMM_MAX], m = -INFINITY;
#pragma unroll
    for (int j = 0; j < ILE_GMM_MAX; j++) {
        const float z = j < g.C ? (u - g.mu[j]) / g.sig[j] : 0.f;
        l[j] = j < g.C ? g.coef[j] - 0.5f * z * z : -INFINITY;
        m = fmaxf(m, l[j]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < ILE_GMM_MAX; j++) s += j < g.C ? expf(l[j] - m) : 0.f;
    lnps = m + logf(s);
    comp = c;
    return u;
}

// z from a standard normal truncated to the box axis with Phi(lo) = p1, Phi(-hi) = q2, mass dm, by
// inverting its CDF at p1 + v dm from the nearer tail (as gmm_draw).
__device__ __forceinline__ float trunc_normal(float p1, float q2, float dm, float v) {
    const float p = p1 + v * dm;
    return p <= 0.5f ? normcdfinvf(p) : -normcdfinvf(q2 + (1.f - v) * dm);
}

// One draw of the sky pair (variables 0, 1) from its correlated mixture: the component is the
// largest c with cw[c] <= a; then attempt t = 0, 1, ... takes Philox block 4 + t of the sample's
// counter, two truncated standard normals y on the component's whitened box and x = mu + L y, and
// keeps the first x inside the rectangle (so the kept x follows the component's normal truncated
// to it).  Returns false after 1024 attempts without one.  ln p_s of the kept x: log-sum-exp of
// coef_c - (x - mu_c)^T cov_c^-1 (x - mu_c) / 2.
__device__ bool pair_draw(const IleSamplerParams &sp, const IleGmm2Tab &g, uint32_t a, uint32_t n, uint32_t iter,
                          float &x0, float &x1, int &comp, float &lnps) {
    int c = 0;
    for (int j = 1; j < g.C; j++)
        if (g.cw[j] <= (uint64_t)a) c = j;
    comp = c;
    const float lo0 = sp.lo[0], hi0 = sp.hi[0], lo1 = sp.lo[1], hi1 = sp.hi[1];
    bool ok = false;
    for (uint32_t t = 0; t < 1024u && !ok; t++) {
        uint32_t w[4];
        philox4x32_10(n, iter, sp.point, 4u + t, sp.key0, sp.key1, w);
        const float y0 = trunc_normal(g.p1[c][0], g.q2[c][0], g.dm[c][0], unit23(w[0]));
        const float y1 = trunc_normal(g.p1[c][1], g.q2[c][1], g.dm[c][1], unit23(w[1]));
        x0 = g.mu[c][0] + g.L[c][0] * y0;
        x1 = g.mu[c][1] + g.L[c][1] * y0 + g.L[c][2] * y1;
        ok = x0 >= lo0 && x0 <= hi0 && x1 >= lo1 && x1 <= hi1;
    }
    if (!ok) {
        x0 = fminf(fmaxf(x0, lo0), hi0);
        x1 = fminf(fmaxf(x1, lo1), hi1);
    }
    float l[ILE_GMM_MAX], m = -INFINITY;
#pragma unroll
    for (int j = 0; j < ILE_GMM_MAX; j++) {
        const float d0 = x0 - g.mu[j][0], d1 = x1 - g.mu[j][1];
        const float q = g.icov[j][0] * d0 * d0 + 2.f * g.icov[j][1] * d0 * d1 + g.icov[j][2] * d1 * d1;
        l[j] = j < g.C ? g.coef[j] - 0.5f * q : -INFINITY;
        m = fmaxf(m, l[j]);
    }
    float sum = 0.f;
#pragma unroll
    for (int j = 0; j < ILE_GMM_MAX; j++) sum += j < g.C ? expf(l[j] - m) : 0.f;
    lnps = m + logf(sum);
    return ok;
}

// Sample n of N (one point): theta [7][N], ln p - ln p_s, bins [7][N].
__device__ __forceinline__ void sample_one(const IleSamplerParams &sp, const SamplerTables &tb, uint32_t iter,
                                           int64_t n, int64_t N, double *__restrict__ theta,
                                           double *__restrict__ lnw_prior, uint8_t *__restrict__ bins,
                                           float *__restrict__ u_gmm, float *__restrict__ u_pair = nullptr,
                                           unsigned *flags = nullptr) {
    const uint32_t(&cdf_s)[ND][NB + 1] = tb.cdf;
    const float(&lnps_s)[ND][NB] = tb.lnps;
    uint32_t wds[16];
#pragma unroll
    for (uint32_t blk = 0; blk < 4; blk++)
        philox4x32_10((uint32_t)n, iter, sp.point, blk, sp.key0, sp.key1, wds + 4 * blk);
    float lw = 0.f;
    float px0 = 0.f, px1 = 0.f;
    int pc = 0;
    if (sp.gmm_pair) {
        // the sky pair together from its correlated mixture; its component uses word 0
        float lnps;
        if (!pair_draw(sp, tb.pair, wds[0], (uint32_t)n, iter, px0, px1, pc, lnps) && flags)
            atomicOr(flags, ILE_FLAG_RANGE);
        lw += -logf(sp.hi[0] - sp.lo[0]) - logf(sp.hi[1] - sp.lo[1]) - lnps;
        u_pair[n] = px0;
        u_pair[N + n] = px1;
    }
#pragma unroll
    for (int d = 0; d < ND; d++) {
        const float lo = sp.lo[d], hi = sp.hi[d];
        const uint32_t a = wds[2 * d], bw = wds[2 * d + 1];
        float u;
        int bin = 255;
        if (sp.gmm_pair && d < 2) {
            u = d == 0 ? px0 : px1;
            bin = pc;
        } else if (sp.gmm_mask & (1u << d)) {
            float lnps;
            u = gmm_draw(tb.gmm[d], lo, hi, a, bw, bin, lnps);
            const float lnp = d == 5 ? logf(3.f * u * u / (hi * hi * hi - lo * lo * lo)) : -logf(hi - lo);
            lw += lnp - lnps;
            u_gmm[(int64_t)__popc(sp.gmm_mask & ((1u << d) - 1u)) * N + n] = u;
        } else if (sp.adapt_mask & (1u << d)) {
            // largest b with cdf[b] <= a (cdf[0] = 0, strictly increasing until 2^32)
            int b0 = 0, b1 = NB;  // invariant: cdf[b0] <= a < cdf[b1] (cdf[100] = 2^32 > a)
            while (b1 - b0 > 1) {
                const int mid = (b0 + b1) >> 1;
                if (cdf_s[d][mid] <= a) b0 = mid; else b1 = mid;
            }
            bin = b0;
            const float width = (hi - lo) * (1.0f / NB);
            u = lo + ((float)bin + unit23(bw)) * width;
            const float lnp = d == 5 ? logf(3.f * u * u / (hi * hi * hi - lo * lo * lo)) : -logf(hi - lo);
            lw += lnp - lnps_s[d][bin];
        } else {
            const float v = unit23(a);
            u = d == 5 ? cbrtf(lo * lo * lo + v * (hi * hi * hi - lo * lo * lo)) : lo + v * (hi - lo);
        }
        float phys = u;
        if (d == 1) phys = asinf(fminf(fmaxf(u, -1.f), 1.f));
        if (d == 3) phys = acosf(fminf(fmaxf(u, -1.f), 1.f));
        if (sp.sky && d == 1) {
            // rotated network frame: (phi', lat') -> Earth-fixed direction -> (ra, dec)
            float sl, cl, sf, cf;
            sincosf(phys, &sl, &cl);
            sincosf((float)theta[n], &sf, &cf);  // phi' was stored at d = 0
            const float a = cl * cf, b = cl * sf;
            const float nx = sp.rot[0] * a + sp.rot[1] * b + sp.rot[2] * sl;
            const float ny = sp.rot[3] * a + sp.rot[4] * b + sp.rot[5] * sl;
            const float nz = sp.rot[6] * a + sp.rot[7] * b + sp.rot[8] * sl;
            float ra = sp.gmst - atan2f(-ny, nx);
            const float twopi = 2.f * ILE_PI_F;
            ra -= twopi * floorf(ra / twopi);
            theta[n] = (double)ra;
            phys = asinf(fminf(fmaxf(nz, -1.f), 1.f));
        }
        theta[(int64_t)d * N + n] = (double)phys;
        bins[(int64_t)d * N + n] = (uint8_t)bin;
    }
    lnw_prior[n] = (double)lw;
}

__global__ void __launch_bounds__(256) sample_kernel(IleSamplerParams sp, const uint64_t *__restrict__ cdf,
                                                     const float *__restrict__ lnps_tab,
                                                     const IleGmmTab *__restrict__ gmm_tab,
                                                     const IleGmm2Tab *__restrict__ pair_tab,
                                                     const int *__restrict__ iter_dev, int64_t N,
                                                     double *__restrict__ theta, double *__restrict__ lnw_prior,
                                                     uint8_t *__restrict__ bins, float *__restrict__ u_gmm,
                                                     float *__restrict__ u_pair, unsigned *flags) {
    __shared__ SamplerTables tb;
    load_tables(tb, cdf, lnps_tab, gmm_tab, sp.gmm_mask, sp.gmm_pair ? pair_tab : nullptr);
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    sample_one(sp, tb, (uint32_t)(*iter_dev), n, N, theta, lnw_prior, bins, u_gmm, u_pair, flags);
}

// Batched: block b draws samples start .. start + 255 of point blk[b].x (blk[b].y = start).
__global__ void __launch_bounds__(256) bsample_kernel(const IleBatchPoint *__restrict__ bp,
                                                      const int2 *__restrict__ blk, const uint64_t *__restrict__ cdf,
                                                      const float *__restrict__ lnps_tab,
                                                      const int *__restrict__ iter_dev, double *__restrict__ theta,
                                                      double *__restrict__ lnw_prior, uint8_t *__restrict__ bins) {
    __shared__ SamplerTables tb;
    const int p = blk[blockIdx.x].x;
    const IleBatchPoint &pt = bp[p];
    load_tables(tb, cdf + (size_t)p * ND * (NB + 1), lnps_tab + (size_t)p * ND * NB, nullptr, 0u);
    __syncthreads();
    const int64_t n = (int64_t)blk[blockIdx.x].y + threadIdx.x;
    if (n >= pt.N) return;
    // batched points use histograms only (sp.gmm_mask = 0)
    sample_one(pt.sp, tb, (uint32_t)iter_dev[p], n, pt.N, theta + ND * pt.off, lnw_prior + pt.off, bins + ND * pt.off,
               nullptr);
}

// Histograms of w_n = exp(ln w_n - max) over each adaptive dimension, as 2^-40 fixed point:
// the lanes of a warp that fall in the same bin are summed first (labelled partition + reduce,
// so an adapted histogram's crowded bins cost one shared atomic per warp, not one per lane), then
// per-block shared-memory integer atomics and one global integer atomic per (d, b) and block.
__device__ __forceinline__ void hist_chunk(const double *__restrict__ lnL, const double *__restrict__ lnw_prior,
                                           const uint8_t *__restrict__ bins, int64_t N, int64_t beg,
                                           const double *__restrict__ iter_res, unsigned mask,
                                           unsigned long long *__restrict__ hist_fx, unsigned long long *h) {
    for (int i = threadIdx.x; i < ND * NB; i += blockDim.x) h[i] = 0ull;
    __syncthreads();
    const double m = iter_res[4];  // max ln w of this iteration
    const int64_t end = min(N, beg + HIST_CHUNK);
    for (int64_t n = beg + threadIdx.x; n < end; n += blockDim.x) {
        const float w = __expf((float)(lnL[n] + lnw_prior[n] - m));
        const unsigned long long wf = (unsigned long long)(w * 1099511627776.0f);  // w * 2^40
#pragma unroll
        for (int d = 0; d < ND; d++) {
            if (mask & (1u << d)) {
                const unsigned b = bins[(int64_t)d * N + n];
                const cg::coalesced_group grp = cg::labeled_partition(cg::coalesced_threads(), b);
                const unsigned long long sum = cg::reduce(grp, wf, cg::plus<unsigned long long>());
                if (grp.thread_rank() == 0 && sum) atomicAdd(&h[d * NB + b], sum);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ND * NB; i += blockDim.x)
        if (h[i]) atomicAdd(&hist_fx[i], h[i]);
}

__global__ void __launch_bounds__(HIST_THREADS) hist_kernel(const double *__restrict__ lnL,
                                                            const double *__restrict__ lnw_prior,
                                                            const uint8_t *__restrict__ bins, int64_t N,
                                                            const double *__restrict__ iter_res, unsigned mask,
                                                            unsigned long long *__restrict__ hist_fx) {
    __shared__ unsigned long long h[ND * NB];
    hist_chunk(lnL, lnw_prior, bins, N, (int64_t)blockIdx.x * HIST_CHUNK, iter_res, mask, hist_fx, h);
}

// Batched: block b takes the HIST_CHUNK samples from blk[b].y of point blk[b].x.
__global__ void __launch_bounds__(HIST_THREADS) bhist_kernel(const IleBatchPoint *__restrict__ bp,
                                                             const int2 *__restrict__ blk,
                                                             const double *__restrict__ lnL,
                                                             const double *__restrict__ lnw_prior,
                                                             const uint8_t *__restrict__ bins,
                                                             const double *__restrict__ iter_res,
                                                             unsigned long long *__restrict__ hist_fx) {
    __shared__ unsigned long long h[ND * NB];
    const int p = blk[blockIdx.x].x;
    const IleBatchPoint &pt = bp[p];
    hist_chunk(lnL + pt.off, lnw_prior + pt.off, bins + ND * pt.off, pt.N, blk[blockIdx.x].y, iter_res + 8 * p,
               pt.sp.adapt_mask, hist_fx + (size_t)p * ND * NB, h);
}

// Next integer tables from the histogram, the ln p_s table, the pooled accumulators and the
// iteration counter.  Threads d < ND build the tables of the adaptive dimensions (sequential
// FP64 accumulation, bit-reproducible); all threads then fill ln p_s.
__device__ __forceinline__ void renorm_point(unsigned long long *__restrict__ hist_fx, unsigned mask, double eps,
                                             const IleSamplerParams &sp, double *__restrict__ hist,
                                             uint64_t *__restrict__ cdf, float *__restrict__ lnps_tab,
                                             const double *__restrict__ iter_res, int64_t N,
                                             double *__restrict__ pooled, double *__restrict__ iter_log,
                                             int *__restrict__ iter_dev, int update_tables) {
    const int i = threadIdx.x;
    __shared__ double hs[ND][NB], tot_s[ND];
    for (int j = i; j < ND * NB; j += blockDim.x) {
        const double v = (double)hist_fx[j] * (1.0 / 1099511627776.0);
        hist[j] = v;
        hs[j / NB][j % NB] = v;
        hist_fx[j] = 0ull;  // ready for the next iteration
    }
    __syncthreads();
    // the bin masses in parallel (FP64 divisions are slow and independent), then the cumulative
    // sums in bin order; the operations and their order are those of the sequential definition
    if (update_tables && i < ND && (mask & (1u << i))) {
        double tot = 0.0;
        for (int b = 0; b < NB; b++) tot = __dadd_rn(tot, hs[i][b]);
        tot_s[i] = tot;
    }
    __syncthreads();
    if (update_tables) {
        const double ome = __dsub_rn(1.0, eps), flo = __ddiv_rn(eps, (double)NB);
        for (int j = i; j < ND * NB; j += blockDim.x) {
            const int d = j / NB, b = j % NB;
            if (mask & (1u << d)) hs[d][b] = __dadd_rn(__dmul_rn(ome, __ddiv_rn(hs[d][b], tot_s[d])), flo);
        }
    }
    __syncthreads();
    if (update_tables && i < ND && (mask & (1u << i))) {
        const int d = i;
        uint64_t *c = cdf + d * (NB + 1);
        double acc = 0.0;
        c[0] = 0;
        for (int b = 0; b < NB; b++) {
            const double mass = hs[d][b];
            acc = __dadd_rn(acc, mass);
            if (b + 1 < NB) {
                double v = floor(__dmul_rn(acc, 4294967296.0));
                if (v > 4294967296.0) v = 4294967296.0;
                c[b + 1] = (uint64_t)v;
            }
        }
        c[NB] = (uint64_t)1 << 32;
        for (int b = 1; b <= NB; b++)
            if (c[b] < c[b - 1]) c[b] = c[b - 1];
    }
    __syncthreads();
    if (update_tables) {
        for (int j = i; j < ND * NB; j += blockDim.x) {
            const int d = j / NB, b = j % NB;
            if (!(mask & (1u << d))) continue;
            const uint64_t *c = cdf + d * (NB + 1);
            const float width = (sp.hi[d] - sp.lo[d]) * (1.0f / NB);
            lnps_tab[j] = logf((float)(c[b + 1] - c[b]) * (1.0f / 4294967296.0f)) - logf(width);
        }
    }
    if (i != 0) return;
    // pooled (m, S1, S2, n) over all iterations, each weighted with its own sampling prior
    const double m_it = iter_res[4], s1_it = iter_res[5], s2_it = iter_res[6];
    const double m_old = pooled[0];
    const double m = fmax(m_old, m_it);
    const double f_old = pooled[3] > 0 ? exp(m_old - m) : 0.0, f_it = exp(m_it - m);
    pooled[1] = pooled[1] * f_old + s1_it * f_it;
    pooled[2] = pooled[2] * f_old * f_old + s2_it * f_it * f_it;
    pooled[0] = m;
    pooled[3] += (double)N;
    const int it = *iter_dev;
    if (it >= 0 && it < ILE_ADAPT_LOG) {
        iter_log[2 * it] = iter_res[0];
        iter_log[2 * it + 1] = iter_res[2];
    }
    *iter_dev = it + 1;
}

__global__ void __launch_bounds__(1024) renorm_kernel(unsigned long long *__restrict__ hist_fx, unsigned mask,
                                                      double eps, IleSamplerParams sp, double *__restrict__ hist,
                                                      uint64_t *__restrict__ cdf, float *__restrict__ lnps_tab,
                                                      const double *__restrict__ iter_res, int64_t N,
                                                      double *__restrict__ pooled, double *__restrict__ iter_log,
                                                      int *__restrict__ iter_dev, int update_tables) {
    renorm_point(hist_fx, mask, eps, sp, hist, cdf, lnps_tab, iter_res, N, pooled, iter_log, iter_dev, update_tables);
}

// Batched: one block per point.
__global__ void __launch_bounds__(1024) brenorm_kernel(const IleBatchPoint *__restrict__ bp,
                                                       unsigned long long *__restrict__ hist_fx,
                                                       double *__restrict__ hist, uint64_t *__restrict__ cdf,
                                                       float *__restrict__ lnps_tab,
                                                       const double *__restrict__ iter_res,
                                                       double *__restrict__ pooled, double *__restrict__ iter_log,
                                                       int *__restrict__ iter_dev) {
    const int p = blockIdx.x;
    const IleBatchPoint &pt = bp[p];
    renorm_point(hist_fx + (size_t)p * ND * NB, pt.sp.adapt_mask, pt.eps, pt.sp, hist + (size_t)p * ND * NB,
                 cdf + (size_t)p * ND * (NB + 1), lnps_tab + (size_t)p * ND * NB, iter_res + 8 * p, pt.N,
                 pooled + 4 * p, iter_log + (size_t)2 * ILE_ADAPT_LOG * p, iter_dev + p, 1);
}

// Uniform tables and the matching ln p_s for every dimension.
__device__ __forceinline__ void reset_point(const IleSamplerParams &sp, uint64_t *__restrict__ cdf,
                                            float *__restrict__ lnps_tab, double *__restrict__ pooled,
                                            int *__restrict__ iter_dev, int iter0) {
    const int i = threadIdx.x;
    for (int j = i; j < ND * (NB + 1); j += blockDim.x) {
        const int b = j % (NB + 1);
        cdf[j] = ((uint64_t)b << 32) / NB;
    }
    __syncthreads();
    for (int j = i; j < ND * NB; j += blockDim.x) {
        const int d = j / NB, b = j % NB;
        const float width = (sp.hi[d] - sp.lo[d]) * (1.0f / NB);
        const uint64_t *c = cdf + d * (NB + 1);
        lnps_tab[j] = logf((float)(c[b + 1] - c[b]) * (1.0f / 4294967296.0f)) - logf(width);
    }
    if (i == 0) {
        pooled[0] = -INFINITY;
        pooled[1] = pooled[2] = pooled[3] = 0.0;
        *iter_dev = iter0;
    }
}

__global__ void reset_kernel(IleSamplerParams sp, uint64_t *__restrict__ cdf, float *__restrict__ lnps_tab,
                             double *__restrict__ pooled, int *__restrict__ iter_dev, int iter0) {
    reset_point(sp, cdf, lnps_tab, pooled, iter_dev, iter0);
}

// Batched: one block per point; also clears the point's histogram accumulators and log.
__global__ void breset_kernel(const IleBatchPoint *__restrict__ bp, uint64_t *__restrict__ cdf,
                              float *__restrict__ lnps_tab, double *__restrict__ pooled, int *__restrict__ iter_dev,
                              unsigned long long *__restrict__ hist_fx, double *__restrict__ hist,
                              double *__restrict__ iter_log) {
    const int p = blockIdx.x;
    for (int j = threadIdx.x; j < ND * NB; j += blockDim.x) {
        hist_fx[(size_t)p * ND * NB + j] = 0ull;
        hist[(size_t)p * ND * NB + j] = 0.0;
    }
    for (int j = threadIdx.x; j < 2 * ILE_ADAPT_LOG; j += blockDim.x) iter_log[(size_t)2 * ILE_ADAPT_LOG * p + j] = 0.0;
    reset_point(bp[p].sp, cdf + (size_t)p * ND * (NB + 1), lnps_tab + (size_t)p * ND * NB, pooled + 4 * p,
                iter_dev + p, 0);
}

// Refresh ln p_s from externally supplied tables (resume).
__global__ void lnps_kernel(IleSamplerParams sp, const uint64_t *__restrict__ cdf, float *__restrict__ lnps_tab) {
    for (int j = threadIdx.x; j < ND * NB; j += blockDim.x) {
        const int d = j / NB, b = j % NB;
        const float width = (sp.hi[d] - sp.lo[d]) * (1.0f / NB);
        const uint64_t *c = cdf + d * (NB + 1);
        lnps_tab[j] = logf((float)(c[b + 1] - c[b]) * (1.0f / 4294967296.0f)) - logf(width);
    }
}

}  // namespace

int ile_hist_partial_count(int64_t N) { return (int)((N + HIST_CHUNK - 1) / HIST_CHUNK); }

cudaError_t ile_launch_sampler_reset(const IleSamplerParams &sp, uint64_t *cdf, float *lnps_tab, double *pooled,
                                     int *iter_dev, int iter0, cudaStream_t st) {
    reset_kernel<<<1, 1024, 0, st>>>(sp, cdf, lnps_tab, pooled, iter_dev, iter0);
    return cudaGetLastError();
}

cudaError_t ile_launch_lnps(const IleSamplerParams &sp, const uint64_t *cdf, float *lnps_tab, cudaStream_t st) {
    lnps_kernel<<<1, 1024, 0, st>>>(sp, cdf, lnps_tab);
    return cudaGetLastError();
}

cudaError_t ile_launch_sample(const IleSamplerParams &sp, const uint64_t *cdf, const float *lnps_tab,
                              const IleGmmTab *gmm_tab, const IleGmm2Tab *pair_tab, const int *iter_dev, int64_t N,
                              double *theta, double *lnw_prior, uint8_t *bins, float *u_gmm, float *u_pair,
                              unsigned *flags, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    if (sp.gmm_mask && (!gmm_tab || !u_gmm)) return cudaErrorInvalidValue;
    if (sp.gmm_pair && (!pair_tab || !u_pair)) return cudaErrorInvalidValue;
    sample_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(sp, cdf, lnps_tab, gmm_tab, pair_tab, iter_dev, N,
                                                               theta, lnw_prior, bins, u_gmm, u_pair, flags);
    return cudaGetLastError();
}

cudaError_t ile_launch_adapt(const double *lnL, const double *lnw_prior, const uint8_t *bins, int64_t N,
                             const double *iter_res, const IleSamplerParams &sp, double eps,
                             unsigned long long *hist_fx, double *hist, uint64_t *cdf, float *lnps_tab, double *pooled,
                             double *iter_log, int *iter_dev, int update_tables, cudaStream_t st) {
    const int np = ile_hist_partial_count(N);
    const unsigned hmask = sp.adapt_mask & ~sp.gmm_mask;  // mixture dimensions adapt in ile_gmm.cu
    hist_kernel<<<np, HIST_THREADS, 0, st>>>(lnL, lnw_prior, bins, N, iter_res, hmask, hist_fx);
    renorm_kernel<<<1, 1024, 0, st>>>(hist_fx, hmask, eps, sp, hist, cdf, lnps_tab, iter_res, N, pooled,
                                      iter_log, iter_dev, update_tables);
    return cudaGetLastError();
}

cudaError_t ile_launch_batch_reset(int n_points, const IleBatchPoint *bp, uint64_t *cdf, float *lnps_tab,
                                   double *pooled, int *iter_dev, unsigned long long *hist_fx, double *hist,
                                   double *iter_log, cudaStream_t st) {
    if (n_points <= 0) return cudaSuccess;
    breset_kernel<<<n_points, 1024, 0, st>>>(bp, cdf, lnps_tab, pooled, iter_dev, hist_fx, hist, iter_log);
    return cudaGetLastError();
}

cudaError_t ile_launch_batch_sample(const IleBatchPoint *bp, const int2 *blk256, int n_blk, const uint64_t *cdf,
                                    const float *lnps_tab, const int *iter_dev, double *theta, double *lnw_prior,
                                    uint8_t *bins, cudaStream_t st) {
    if (n_blk <= 0) return cudaSuccess;
    bsample_kernel<<<n_blk, 256, 0, st>>>(bp, blk256, cdf, lnps_tab, iter_dev, theta, lnw_prior, bins);
    return cudaGetLastError();
}

int ile_hist_chunk() { return HIST_CHUNK; }

cudaError_t ile_launch_batch_adapt(int n_points, const IleBatchPoint *bp, const int2 *hblk, int n_hblk,
                                   const double *lnL, const double *lnw_prior, const uint8_t *bins,
                                   const double *iter_res, unsigned long long *hist_fx, double *hist, uint64_t *cdf,
                                   float *lnps_tab, double *pooled, double *iter_log, int *iter_dev,
                                   cudaStream_t st) {
    if (n_hblk > 0)
        bhist_kernel<<<n_hblk, HIST_THREADS, 0, st>>>(bp, hblk, lnL, lnw_prior, bins, iter_res, hist_fx);
    brenorm_kernel<<<n_points, 1024, 0, st>>>(bp, hist_fx, hist, cdf, lnps_tab, iter_res, pooled, iter_log, iter_dev);
    return cudaGetLastError();
}

extern "C" ile_status ile_philox4x32_10(const uint32_t *ctr_key, int64_t n, uint32_t *out, void *cuda_stream) {
    if (!ctr_key || !out || n < 1 || n > (1ll << 24)) return ILE_E_ARG;
    philox_kat_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(ctr_key, n, out);
    return cudaGetLastError() == cudaSuccess ? ILE_OK : ILE_E_CUDA;
}
