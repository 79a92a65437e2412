// ile_sort.cu -- orders the extrinsic samples so that a 128-sample tile needs few time columns.
//
// A sample's window start in detector k is t_c f_s + dt_k f_s + const, and the light-travel
// delays dt_k (up to ~87 bins at 4096 Hz) dominate the spread between samples.  The delays are
// smooth functions of the source direction in the Earth-fixed frame, so samples are bucketed by
// sky cell: a 128 x 128 grid in (Earth-fixed longitude gmst - ra, sin dec), cells ordered along a
// Hilbert curve so that consecutive buckets are neighbouring cells.  Counting sort: count ->
// exclusive scan -> scatter.  Within a bucket the order is whatever the atomics give; no result
// depends on it, because every sample is evaluated independently and the Monte Carlo sums run
// over the caller's order.
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
