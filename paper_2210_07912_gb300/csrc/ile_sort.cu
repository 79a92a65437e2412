// ile_sort.cu -- orders the extrinsic samples so that a 128-sample tile needs few time columns.
//
// A sample's window start in detector k is t_c f_s + dt_k f_s + const, and the light-travel
// delays dt_k (up to ~87 bins at 4096 Hz) dominate the spread between samples.  The delays are
// smooth functions of the source direction in the Earth-fixed frame, so samples are bucketed by
// sky cell: a 128 x 128 grid in (Earth-fixed longitude gmst - ra, sin dec), cells ordered along a
// Hilbert curve so that consecutive buckets are neighbouring cells.  Counting sort: count ->
// exclusive scan -> scatter.  Within a bucket the order is whatever the atomics give; no result of
// the forward pass depends on it, because every sample is evaluated independently and the Monte
// Carlo sums run over the caller's order.
//
// The adjoint's dQ sums over samples in processing order (FP32 partial sums per chunk of 32), so
// the gradient takes the stable form: a two-pass LSD radix sort of the same 14-bit keys (7 bits
// per pass), each pass a per-block digit histogram, an exclusive scan of the histograms in
// (digit, block) order and a scatter that ranks a block's samples among equal digits in index
// order (warp match, then a prefix over the block's warps, round by round).  Equal keys keep the
// caller's order, so the permutation, and every sum taken in its order, is the same on every run.
#include "ile_internal.cuh"

namespace {

constexpr int GRID = 128;  // cells per axis
constexpr int NKEY = GRID * GRID;

// Hilbert-curve index of cell (x, y) on a GRID x GRID grid.
__device__ __forceinline__ int hilbert_index(int x, int y) {
    int d = 0;
    for (int s = GRID / 2; s > 0; s >>= 1) {
        const int rx = (x & s) ? 1 : 0, ry = (y & s) ? 1 : 0;
        d += s * s * ((3 * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = s - 1 - x;
                y = s - 1 - y;
            }
            const int tmp = x;
            x = y;
            y = tmp;
        }
    }
    return d;
}

__device__ __forceinline__ int delay_key(float gmst, const double *__restrict__ samples, int64_t N, int64_t n) {
    const double ra = samples[n], dec = samples[N + n];
    float lon = (float)(gmst - ra) * (1.0f / (2.0f * ILE_PI_F));
    lon -= floorf(lon);
    const float sd = 0.5f * (sinf((float)dec) + 1.0f);
    // fminf/fmaxf also map NaN to a valid cell: non-finite samples are flagged elsewhere
    const int x = (int)fminf(fmaxf(lon * GRID, 0.f), (float)(GRID - 1));
    const int y = (int)fminf(fmaxf(sd * GRID, 0.f), (float)(GRID - 1));
    return hilbert_index(x, y);
}

__global__ void __launch_bounds__(256) key_count_kernel(const __grid_constant__ PointParams pp,
                                                        const double *__restrict__ samples, int64_t N,
                                                        int *__restrict__ keys, int *__restrict__ count) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int key = delay_key(pp.gmst, samples, N, n);
    keys[n] = key;
    atomicAdd(&count[key], 1);
}

// Exclusive scan of NKEY counts in one block of 1024 threads: warp w scans the contiguous segment
// [w * SEG, (w + 1) * SEG) in 32-element rows read and written coalesced (lane l holds element
// i * 32 + l of its segment), after a scan of the 32 segment totals.
constexpr int SEG = NKEY / 32;
static_assert(NKEY % 1024 == 0, "scan layout");
// (one block per point in the batched form: block b scans count + b * NKEY)
__global__ void __launch_bounds__(1024) scan_kernel(int *__restrict__ count) {
    constexpr int ROWS = SEG / 32;
    __shared__ int warp_tot[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    int *c = count + (size_t)blockIdx.x * NKEY + (size_t)warp * SEG;
    int v[ROWS];
    int tot = 0;
#pragma unroll
    for (int i = 0; i < ROWS; i++) {
        v[i] = c[i * 32 + lane];
        tot += v[i];
    }
    for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) warp_tot[warp] = tot;
    __syncthreads();
    if (warp == 0) {
        const int x = warp_tot[lane];
        int incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        warp_tot[lane] = incl - x;  // exclusive: counts before segment `lane`
    }
    __syncthreads();
    int carry = warp_tot[warp];
#pragma unroll
    for (int i = 0; i < ROWS; i++) {
        int incl = v[i];
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        c[i * 32 + lane] = carry + incl - v[i];
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

__global__ void __launch_bounds__(256) scatter_kernel(const int *__restrict__ keys, int64_t N, int *__restrict__ cursor,
                                                      int *__restrict__ perm) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int pos = atomicAdd(&cursor[keys[n]], 1);
    perm[pos] = (int)n;
}

// Batched: block b keys samples blk[b].y .. + 255 of point blk[b].x (local indices; bucket
// counts and keys per point).
__global__ void __launch_bounds__(256) bkey_count_kernel(const IleBatchPoint *__restrict__ bp,
                                                         const int2 *__restrict__ blk,
                                                         const double *__restrict__ theta, int *__restrict__ keys,
                                                         int *__restrict__ count) {
    const int p = blk[blockIdx.x].x;
    const IleBatchPoint &pt = bp[p];
    const int64_t n = (int64_t)blk[blockIdx.x].y + threadIdx.x;
    if (n >= pt.N) return;
    const int key = delay_key(pt.gmst, theta + ILE_NDIM * pt.off, pt.N, n);
    keys[pt.off + n] = key;
    atomicAdd(&count[(size_t)p * NKEY + key], 1);
}

__global__ void __launch_bounds__(256) bscatter_kernel(const IleBatchPoint *__restrict__ bp,
                                                       const int2 *__restrict__ blk, const int *__restrict__ keys,
                                                       int *__restrict__ cursor, int *__restrict__ perm) {
    const int p = blk[blockIdx.x].x;
    const IleBatchPoint &pt = bp[p];
    const int64_t n = (int64_t)blk[blockIdx.x].y + threadIdx.x;
    if (n >= pt.N) return;
    const int pos = atomicAdd(&cursor[(size_t)p * NKEY + keys[pt.off + n]], 1);
    perm[pt.off + pos] = (int)n;
}

}  // namespace

size_t ile_sort_key_buckets() { return NKEY; }

cudaError_t ile_launch_batch_sort(int n_points, const IleBatchPoint *bp, const int2 *blk256, int n_blk,
                                  const double *theta, int *keys, int *buckets, int *perm, cudaStream_t st) {
    if (n_blk <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(buckets, 0, sizeof(int) * NKEY * (size_t)n_points, st);
    if (e != cudaSuccess) return e;
    bkey_count_kernel<<<n_blk, 256, 0, st>>>(bp, blk256, theta, keys, buckets);
    scan_kernel<<<n_points, 1024, 0, st>>>(buckets);
    bscatter_kernel<<<n_blk, 256, 0, st>>>(bp, blk256, keys, buckets, perm);
    return cudaGetLastError();
}

namespace {

// ---------------------------------------------------------------- stable (deterministic) form
constexpr int SS_T = 256;              // threads per block
constexpr int SS_PER = 4;              // samples per thread (rounds of 256 in index order)
constexpr int SS_BLK = SS_T * SS_PER;  // samples per block
constexpr int RDX = 128;               // 7-bit digits; two passes cover the 14-bit keys
static_assert(RDX * RDX == NKEY, "two 7-bit digits per key");

// per-block histogram of digit (key >> shift) & (RDX - 1), written digit-major: hist[d * nblk + b];
// with samples given, the keys are formed here (pass 1) and stored
__global__ void __launch_bounds__(SS_T) ss_hist_kernel(const __grid_constant__ PointParams pp,
                                                       const double *__restrict__ samples, int *__restrict__ keys,
                                                       int64_t N, int shift, int *__restrict__ hist, int nblk) {
    __shared__ int h[RDX];
    for (int i = threadIdx.x; i < RDX; i += SS_T) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SS_BLK;
    for (int r = 0; r < SS_PER; r++) {
        const int64_t n = base + (int64_t)r * SS_T + threadIdx.x;
        if (n >= N) break;
        int key;
        if (samples) {
            key = delay_key(pp.gmst, samples, N, n);
            keys[n] = key;
        } else {
            key = keys[n];
        }
        atomicAdd(&h[(key >> shift) & (RDX - 1)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RDX; i += SS_T) hist[(size_t)i * nblk + blockIdx.x] = h[i];
}

// exclusive scan of L counts in place, one block of 1024 threads, in pages of 32 warps x SC_ROWS
// rows of 32: warp w scans the contiguous segment [w * 32 SC_ROWS, (w + 1) * 32 SC_ROWS) of the
// page in 32-element rows read and written coalesced (lane l holds element 32 i + l), after a scan
// of the 32 segment totals (the layout of scan_kernel, with a carry from page to page)
constexpr int SC_ROWS = 32;
__global__ void __launch_bounds__(1024) ss_scan_kernel(int *__restrict__ a, int L) {
    __shared__ int wsum[32];
    __shared__ int page_tot;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    int carry = 0;
    for (int p0 = 0; p0 < L; p0 += 1024 * SC_ROWS) {
        const int sb = p0 + warp * 32 * SC_ROWS;
        int v[SC_ROWS];
        int tot = 0;
#pragma unroll
        for (int i = 0; i < SC_ROWS; i++) {
            const int e = sb + 32 * i + lane;
            v[i] = e < L ? a[e] : 0;
            tot += v[i];
        }
        for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        if (lane == 0) wsum[warp] = tot;
        __syncthreads();
        if (warp == 0) {
            const int x = wsum[lane];
            int wi = x;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += u;
            }
            wsum[lane] = wi - x;  // counts of the page before segment `lane`
            if (lane == 31) page_tot = wi;
        }
        __syncthreads();
        int run = carry + wsum[warp];
#pragma unroll
        for (int i = 0; i < SC_ROWS; i++) {
            int incl = v[i];
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            const int e = sb + 32 * i + lane;
            if (e < L) a[e] = run + incl - v[i];
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        carry += page_tot;
        __syncthreads();  // wsum and page_tot are rewritten by the next page
    }
}

// stable scatter of one pass: the sample at index n of this block goes to off(d, block) + (the
// number of the block's samples before n with the same digit d).  vin null: the values are the
// indices n themselves; kout null: keys are not written.
__global__ void __launch_bounds__(SS_T) ss_scatter_kernel(const int *__restrict__ kin, const int *__restrict__ vin,
                                                          int64_t N, int shift, const int *__restrict__ off, int nblk,
                                                          int *__restrict__ kout, int *__restrict__ vout) {
    __shared__ int run[RDX];
    __shared__ int cnt[SS_T / 32][RDX];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < RDX; i += SS_T) run[i] = off[(size_t)i * nblk + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * SS_BLK;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < SS_PER; r++) {
        if (base + (int64_t)r * SS_T >= N) break;  // uniform over the block
        for (int i = tid; i < (SS_T / 32) * RDX; i += SS_T) (&cnt[0][0])[i] = 0;
        __syncthreads();
        const int64_t n = base + (int64_t)r * SS_T + tid;
        const bool valid = n < N;
        const int key = valid ? kin[n] : 0;
        const int d = valid ? (key >> shift) & (RDX - 1) : RDX;  // past-the-end lanes form their own group
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) cnt[warp][d] = __popc(peers);
        __syncthreads();
        if (tid < RDX) {
            int acc = run[tid];
#pragma unroll
            for (int w = 0; w < SS_T / 32; w++) {
                const int c = cnt[w][tid];
                cnt[w][tid] = acc;
                acc += c;
            }
            run[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            const int pos = cnt[warp][d] + rank;
            if (kout) kout[pos] = key;
            vout[pos] = vin ? vin[n] : (int)n;
        }
        __syncthreads();  // cnt is cleared for the next round
    }
}

}  // namespace

size_t ile_sort_stable_work_ints(int64_t N) {
    const int64_t nblk = (N + SS_BLK - 1) / SS_BLK;
    return (size_t)(2 * N + (int64_t)RDX * nblk);
}

cudaError_t ile_launch_sort_stable(const PointParams &pp, const double *samples, int64_t N, int *keys, int *work,
                                   int *perm, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const int nblk = (int)((N + SS_BLK - 1) / SS_BLK);
    int *k1 = work, *v1 = work + N, *hist = work + 2 * N;
    const int L = RDX * nblk;
    // pass 1: low 7 bits, from the caller's order
    ss_hist_kernel<<<nblk, SS_T, 0, st>>>(pp, samples, keys, N, 0, hist, nblk);
    ss_scan_kernel<<<1, 1024, 0, st>>>(hist, L);
    ss_scatter_kernel<<<nblk, SS_T, 0, st>>>(keys, nullptr, N, 0, hist, nblk, k1, v1);
    // pass 2: high 7 bits, stable over pass 1's order
    ss_hist_kernel<<<nblk, SS_T, 0, st>>>(pp, nullptr, k1, N, 7, hist, nblk);
    ss_scan_kernel<<<1, 1024, 0, st>>>(hist, L);
    ss_scatter_kernel<<<nblk, SS_T, 0, st>>>(k1, v1, N, 7, hist, nblk, nullptr, perm);
    return cudaGetLastError();
}

cudaError_t ile_launch_sort(const PointParams &pp, const double *samples, int64_t N, int *keys, int *buckets,
                            int *perm, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(buckets, 0, sizeof(int) * NKEY, st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    key_count_kernel<<<blocks, 256, 0, st>>>(pp, samples, N, keys, buckets);
    scan_kernel<<<1, 1024, 0, st>>>(buckets);
    scatter_kernel<<<blocks, 256, 0, st>>>(keys, N, buckets, perm);
    return cudaGetLastError();
}
