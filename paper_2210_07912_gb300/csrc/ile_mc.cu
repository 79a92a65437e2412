// ile_mc.cu -- stage S6: Monte Carlo marginal likelihood of Eq. (eq:lnL:MonteCarlo) in log space.
//
// ln w_n = lnL_t(n) + ln p(theta_n) - ln p_s(theta_n).  Each block reduces one contiguous chunk to
// a partial (max ln w, S1 = sum e^{ln w - max}, S2 = sum e^{2(ln w - max)}) -- exponentials and
// sums in FP64, relative to the block maximum -- and a one-block merge combines the
// partials in a fixed tree order, so the result does not depend on scheduling.  The merge gives
//   ln I = max + ln(S1/N),  sigma_ln = sigma_I / I = sqrt((N S2/S1^2 - 1)/(N - 1)),
//   n_eff = S1 (= sum w / max w, Eq. (eq:neff)),  ess = S1^2 / S2 (Eq. (eq:neff_ESS)).
#include "ile_internal.cuh"

namespace {

constexpr int MC_THREADS = 256;
constexpr int MC_CHUNK = 4096;
constexpr int MC_MAX_PART = 4096;

__device__ __forceinline__ double lnw_at(const double *lnL, const double *lp, const double *lps, int64_t n) {
    double v = lnL[n];
    if (lp) v += lp[n];
    if (lps) v -= lps[n];
    return v;
}

template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    T r = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) r = op(r, sh[w]);
    return r;
}

__device__ __forceinline__ void mc_partial_chunk(const double *__restrict__ lnL, const double *__restrict__ lp,
                                                 const double *__restrict__ lps, int64_t N, int64_t beg,
                                                 double *__restrict__ part, double *sh) {
    const int64_t end = min(N, beg + MC_CHUNK);
    double m = -INFINITY;
    for (int64_t n = beg + threadIdx.x; n < end; n += MC_THREADS) m = fmax(m, lnw_at(lnL, lp, lps, n));
    m = block_reduce(m, [](double a, double b) { return fmax(a, b); }, sh);
    double s1 = 0.0, s2 = 0.0;
    for (int64_t n = beg + threadIdx.x; n < end; n += MC_THREADS) {
        const double e = exp(lnw_at(lnL, lp, lps, n) - m);
        s1 += e;
        s2 += e * e;
    }
    s1 = block_reduce(s1, [](double a, double b) { return a + b; }, sh);
    s2 = block_reduce(s2, [](double a, double b) { return a + b; }, sh);
    if (threadIdx.x == 0) {
        part[0] = m;
        part[1] = s1;
        part[2] = s2;
    }
}

__global__ void __launch_bounds__(MC_THREADS) mc_partial_kernel(const double *__restrict__ lnL,
                                                                const double *__restrict__ lp,
                                                                const double *__restrict__ lps, int64_t N,
                                                                double *__restrict__ part) {
    __shared__ double sh[MC_THREADS / 32];
    mc_partial_chunk(lnL, lp, lps, N, (int64_t)blockIdx.x * MC_CHUNK, part + 3 * blockIdx.x, sh);
}

__device__ __forceinline__ void mc_merge_body(const double *__restrict__ part, int n_part, int64_t N,
                                              double *__restrict__ result, double *sh) {
    double m = -INFINITY;
    for (int b = threadIdx.x; b < n_part; b += MC_THREADS) m = fmax(m, part[3 * b]);
    m = block_reduce(m, [](double a, double b) { return fmax(a, b); }, sh);
    double s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < n_part; b += MC_THREADS) {
        const double f = exp(part[3 * b] - m);
        s1 += part[3 * b + 1] * f;
        s2 += part[3 * b + 2] * f * f;
    }
    s1 = block_reduce(s1, [](double a, double b) { return a + b; }, sh);
    s2 = block_reduce(s2, [](double a, double b) { return a + b; }, sh);
    if (threadIdx.x != 0) return;
    const double Nd = (double)N;
    const double mean = s1 / Nd;
    double var = (s2 - Nd * mean * mean) / (Nd - 1.0);
    if (var < 0.0) var = 0.0;
    result[0] = m + log(mean);
    result[1] = N > 1 ? sqrt(var / Nd) / mean : INFINITY;
    result[2] = s1;
    result[3] = s1 * s1 / s2;
    result[4] = m;
    result[5] = s1;
    result[6] = s2;
}

__global__ void __launch_bounds__(MC_THREADS) mc_merge_kernel(const double *__restrict__ part, int n_part, int64_t N,
                                                              double *__restrict__ result) {
    __shared__ double sh[MC_THREADS / 32];
    mc_merge_body(part, n_part, N, result, sh);
}

// Batched (adaptive run: ln w = lnL_t + (ln p - ln p_s)): block b reduces chunk b, which is
// samples mblk[b].y .. + MC_CHUNK of point mblk[b].x; the merge takes one block per point over
// its chunks mblk_first[p] .. mblk_first[p + 1].
__global__ void __launch_bounds__(MC_THREADS) bmc_partial_kernel(const IleBatchPoint *__restrict__ bp,
                                                                 const int2 *__restrict__ mblk,
                                                                 const double *__restrict__ lnL,
                                                                 const double *__restrict__ lnwp,
                                                                 double *__restrict__ part) {
    __shared__ double sh[MC_THREADS / 32];
    const IleBatchPoint &pt = bp[mblk[blockIdx.x].x];
    mc_partial_chunk(lnL + pt.off, lnwp + pt.off, nullptr, pt.N, mblk[blockIdx.x].y, part + 3 * blockIdx.x, sh);
}

__global__ void __launch_bounds__(MC_THREADS) bmc_merge_kernel(const IleBatchPoint *__restrict__ bp,
                                                               const int *__restrict__ first,
                                                               const double *__restrict__ part,
                                                               double *__restrict__ iter_res) {
    __shared__ double sh[MC_THREADS / 32];
    const int p = blockIdx.x;
    mc_merge_body(part + 3 * first[p], first[p + 1] - first[p], bp[p].N, iter_res + 8 * p, sh);
}

// d ln I / d lnL_t(n) = w_n / sum w = exp(ln w_n - max) / S1 (the derivative of Eq. (eq:lnL:MonteCarlo)
// in log space), with max and S1 from the merged result.
// The upstream scalar is *scale_dev when given (a device pointer), else scale.
__global__ void mc_weights_kernel(const double *__restrict__ lnL, const double *__restrict__ lp,
                                  const double *__restrict__ lps, int64_t N, const double *__restrict__ result,
                                  const double *__restrict__ scale_dev, double scale, double *__restrict__ g) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double sc = scale_dev ? *scale_dev : scale;
    g[n] = sc * exp(lnw_at(lnL, lp, lps, n) - result[4]) / result[5];
}

}  // namespace

int ile_mc_chunk() { return MC_CHUNK; }

cudaError_t ile_launch_batch_mc(int n_points, const IleBatchPoint *bp, const int2 *mblk, int n_mblk,
                                const int *mblk_first, const double *lnL, const double *lnw_prior, double *partials,
                                double *iter_res, cudaStream_t st) {
    if (n_mblk <= 0) return cudaSuccess;
    bmc_partial_kernel<<<n_mblk, MC_THREADS, 0, st>>>(bp, mblk, lnL, lnw_prior, partials);
    bmc_merge_kernel<<<n_points, MC_THREADS, 0, st>>>(bp, mblk_first, partials, iter_res);
    return cudaGetLastError();
}

int ile_mc_partial_count(int64_t N) {
    int64_t p = (N + MC_CHUNK - 1) / MC_CHUNK;
    return (int)(p < 1 ? 1 : p);
}

cudaError_t ile_launch_mc(const double *lnL_t, const double *ln_prior, const double *ln_ps, int64_t N,
                          double *partials, int n_part, double *result, cudaStream_t st) {
    if (N <= 0 || n_part != ile_mc_partial_count(N) || n_part > MC_MAX_PART * 1024) return cudaErrorInvalidValue;
    mc_partial_kernel<<<n_part, MC_THREADS, 0, st>>>(lnL_t, ln_prior, ln_ps, N, partials);
    mc_merge_kernel<<<1, MC_THREADS, 0, st>>>(partials, n_part, N, result);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ allocation-free variant
//
// ile_mc_reduce_noalloc runs the same two kernels with their per-block partial sums in a
// file-scope device array instead of context-owned memory, for callers that may not allocate
// device memory (see include/ile.h).  The array exists on every device that loads the library,
// for as long as the CUDA context that loaded it (normally until the process exits).  Host code
// must not pass the symbol itself to a kernel (on the host it is only a stand-in); its device
// address is looked up with cudaGetSymbolAddress on every call, so a context rebuilt by
// cudaDeviceReset gets the new array's address rather than a stale one.

namespace {

constexpr int NOALLOC_MAX_PART = ILE_NOALLOC_MAX_SAMPLES / MC_CHUNK;
static_assert(ILE_NOALLOC_MAX_SAMPLES % MC_CHUNK == 0, "scratch sizing");

static __device__ __align__(256) double g_noalloc_partials[3 * NOALLOC_MAX_PART];

}  // namespace

extern "C" ile_status ile_mc_reduce_noalloc(const double *lnL_t, const double *ln_prior, const double *ln_ps,
                                            int64_t N, double *result, void *cuda_stream) {
    if (!lnL_t || !result || N < 1) return ILE_E_ARG;
    if (N > ILE_NOALLOC_MAX_SAMPLES) return ILE_E_ARG;  // the fixed scratch holds this many samples' partials
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return ILE_E_CUDA;
    double *part = static_cast<double *>(p);
    // every partial the merge reads is written by the partial kernel of the same call, so the
    // shared array needs no clearing between calls
    const int np = ile_mc_partial_count(N);
    if (ile_launch_mc(lnL_t, ln_prior, ln_ps, N, part, np, result, (cudaStream_t)cuda_stream) != cudaSuccess)
        return ILE_E_CUDA;
    return ILE_OK;
}

cudaError_t ile_launch_mc_weights(const double *lnL_t, const double *ln_prior, const double *ln_ps, int64_t N,
                                  const double *result, const double *scale_dev, double scale, double *g,
                                  cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    mc_weights_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(lnL_t, ln_prior, ln_ps, N, result, scale_dev,
                                                                   scale, g);
    return cudaGetLastError();
}
