// ile_sort.cu -- orders the extrinsic samples so that a 128-sample tile needs few time columns.
//
// A sample's window start in detector k is t_c f_s + dt_k f_s + const, and the light-travel
// delays dt_k (up to ~87 bins at 4096 Hz) dominate the spread between samples.  Samples are
// bucketed by their quantised delays (dt_k f_s / 4 for the first three detectors, 64 levels
// each, lexicographic key) with a counting sort: count -> exclusive scan -> scatter.  Within a
// bucket the order is whatever the atomics give; no result depends on it, because every sample
// is evaluated independently and the Monte Carlo sums run over the original order.
#include "ile_internal.cuh"

namespace {

constexpr int KEY_BITS = 6;
constexpr int NKEY = 1 << (3 * KEY_BITS);

__device__ __forceinline__ int delay_key(const PointParams &pp, const double *__restrict__ samples, int64_t N,
                                         int64_t n) {
    const float ra = (float)samples[n], dec = (float)samples[N + n];
    float sg, cg, sd, cd;
    sincosf(pp.gmst - ra, &sg, &cg);
    sincosf(dec, &sd, &cd);
    const float n0 = cd * cg, n1 = -cd * sg, n2 = sd;
    int key = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        int q = 0;
        if (k < pp.K) {
            float dt = -(pp.det_pos_c[k][0] * n0 + pp.det_pos_c[k][1] * n1 + pp.det_pos_c[k][2] * n2) * pp.fs;
            float v = floorf(dt * 0.25f) + 32.f;
            v = fminf(fmaxf(v, 0.f), 63.f);  // also maps NaN to 0: non-finite samples are flagged elsewhere
            q = (int)v;
        }
        key = (key << KEY_BITS) | q;
    }
    return key;
}

__global__ void __launch_bounds__(256) key_count_kernel(const __grid_constant__ PointParams pp,
                                                        const double *__restrict__ samples, int64_t N,
                                                        int *__restrict__ keys, int *__restrict__ count) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int key = delay_key(pp, samples, N, n);
    keys[n] = key;
    atomicAdd(&count[key], 1);
}

// Exclusive scan of NKEY counts in one block of 1024 threads (NKEY / 1024 entries per thread).
__global__ void __launch_bounds__(1024) scan_kernel(int *__restrict__ count) {
    constexpr int PER = NKEY / 1024;
    __shared__ int warp_tot[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    int *c = count + t * PER;
    int local = 0;
    for (int i = 0; i < PER; i++) local += c[i];
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = warp_tot[lane];
        int vi = v;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += u;
        }
        warp_tot[lane] = vi - v;
    }
    __syncthreads();
    int run = warp_tot[warp] + incl - local;
    for (int i = 0; i < PER; i++) {
        int v = c[i];
        c[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(256) scatter_kernel(const int *__restrict__ keys, int64_t N, int *__restrict__ cursor,
                                                      int *__restrict__ perm) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int pos = atomicAdd(&cursor[keys[n]], 1);
    perm[pos] = (int)n;
}

}  // namespace

size_t ile_sort_key_buckets() { return NKEY; }

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
