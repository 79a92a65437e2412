// ile_quv.cu -- the inner-product arrays of Eq. (eq:QUV) from mode waveforms, PSDs and data, on
// the device in FP64 (the step that produces an intrinsic point's Q, U, V):
//   Q_k,a(t) = 2 df sum_m e^{2 pi i f_m t} conj(h_a(f_m)) d_k(f_m) / S_k(f_m)
//   U_k,ab   = 2 df sum_m conj(h_a(f_m)) h_b(f_m) / S_k(f_m)
//   V_k,ab   = 2 df sum_m h_a(-f_m) h_b(f_m) / S_k(f_m)          (<h_a^*|h_b>: FT of conj(h_a(t)))
// over the bins with |f_m| > f_low of a two-sided series in FFT order (f_m = m df for
// m < L/2, (m - L) df otherwise), at t = t_start + i / fs, i < T_ext.
//
// Kernels: quv_weights forms z_k,a(m) = 2 df conj(h_a) d_k / S_k (zero below f_low);
// quv_uv reduces one (k, a, b) entry of U and V per block; quv_q gives each thread one output
// time and walks the frequencies with a rotating phasor e^{2 pi i f_m t} (one sincos per thread,
// FP64 recurrence), the weights staged through shared memory in chunks.
#include "ile_internal.cuh"

namespace {

constexpr int QCH = 512;  // frequencies per staged chunk

__device__ __forceinline__ double freq_of(int64_t m, int64_t L, double df) { return (m < L / 2 ? m : m - L) * df; }

__global__ void quv_weights_kernel(int K, int M, int64_t L, const double2 *__restrict__ h, const double *__restrict__ psd,
                                   const double2 *__restrict__ d, double df, double f_low, double2 *__restrict__ z) {
    const int64_t total = (int64_t)K * M * L;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i % L;
        const int a = (int)((i / L) % M), k = (int)(i / (L * M));
        double2 v = make_double2(0.0, 0.0);
        if (fabs(freq_of(m, L, df)) > f_low) {
            const double2 ha = h[(int64_t)a * L + m], dk = d[(int64_t)k * L + m];
            const double w = 2.0 * df / psd[(int64_t)k * L + m];
            v.x = w * (ha.x * dk.x + ha.y * dk.y);  // conj(h) d
            v.y = w * (ha.x * dk.y - ha.y * dk.x);
        }
        z[i] = v;
    }
}

template <typename T>
__device__ T block_sum(T v, T *sh) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    T r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += sh[w];
    return r;
}

__global__ void __launch_bounds__(256) quv_uv_kernel(int M, int64_t L, const double2 *__restrict__ h,
                                                     const double *__restrict__ psd, double df, double f_low,
                                                     double2 *__restrict__ U, double2 *__restrict__ V) {
    __shared__ double sh[8];
    const int b = blockIdx.x % M, a = (blockIdx.x / M) % M, k = blockIdx.x / (M * M);
    double ur = 0.0, ui = 0.0, vr = 0.0, vi = 0.0;
    for (int64_t m = threadIdx.x; m < L; m += blockDim.x) {
        if (!(fabs(freq_of(m, L, df)) > f_low)) continue;
        const double w = 2.0 * df / psd[(int64_t)k * L + m];
        const double2 ha = h[(int64_t)a * L + m], hb = h[(int64_t)b * L + m];
        const double2 hm = h[(int64_t)a * L + (m == 0 ? 0 : L - m)];  // h_a(-f_m)
        ur += w * (ha.x * hb.x + ha.y * hb.y);
        ui += w * (ha.x * hb.y - ha.y * hb.x);
        vr += w * (hm.x * hb.x - hm.y * hb.y);
        vi += w * (hm.x * hb.y + hm.y * hb.x);
    }
    ur = block_sum(ur, sh);
    ui = block_sum(ui, sh);
    vr = block_sum(vr, sh);
    vi = block_sum(vi, sh);
    if (threadIdx.x == 0) {
        U[blockIdx.x] = make_double2(ur, ui);
        V[blockIdx.x] = make_double2(vr, vi);
    }
}

// grid: (ceil(T_ext / 128), K * M); 128 threads, one output time each
__global__ void __launch_bounds__(128) quv_q_kernel(int64_t L, const double2 *__restrict__ z, double df,
                                                    double t_start, double fs, int T_ext, double2 *__restrict__ Q) {
    __shared__ double2 zs[QCH];
    const int series = blockIdx.y;
    const int i = blockIdx.x * 128 + threadIdx.x;
    const double t = t_start + (double)i / fs;
    const double2 *zz = z + (int64_t)series * L;
    double accr = 0.0, acci = 0.0;
    for (int64_t m0 = 0; m0 < L; m0 += QCH) {
        const int n = (int)min((int64_t)QCH, L - m0);
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += 128) zs[j] = zz[m0 + j];
        __syncthreads();
        // phasor at the chunk's first frequency, then the per-bin step (frequencies are
        // consecutive within a chunk except across the Nyquist wrap, where it restarts)
        double s0, c0, s1, c1;
        sincospi(2.0 * freq_of(m0, L, df) * t, &s0, &c0);
        sincospi(2.0 * df * t, &s1, &c1);
        double wr = c0, wi = s0;
        for (int j = 0; j < n; j++) {
            const int64_t m = m0 + j;
            if (m == L / 2 && j > 0) sincospi(2.0 * freq_of(m, L, df) * t, &wi, &wr);
            const double2 v = zs[j];
            accr += v.x * wr - v.y * wi;
            acci += v.x * wi + v.y * wr;
            const double nr = wr * c1 - wi * s1;
            wi = wr * s1 + wi * c1;
            wr = nr;
        }
    }
    if (i < T_ext) Q[(int64_t)series * T_ext + i] = make_double2(accr, acci);
}

}  // namespace

cudaError_t ile_launch_quv(int K, int M, int64_t L, const double *h, const double *psd, const double *d, double df,
                           double f_low, double t_start, double fs, int T_ext, double *z, double *Q, double *U,
                           double *V, cudaStream_t st) {
    quv_weights_kernel<<<1024, 256, 0, st>>>(K, M, L, (const double2 *)h, psd, (const double2 *)d, df, f_low,
                                             (double2 *)z);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    quv_uv_kernel<<<K * M * M, 256, 0, st>>>(M, L, (const double2 *)h, psd, df, f_low, (double2 *)U, (double2 *)V);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((T_ext + 127) / 128, K * M);
    quv_q_kernel<<<grid, 128, 0, st>>>(L, (const double2 *)z, df, t_start, fs, T_ext, (double2 *)Q);
    return cudaGetLastError();
}
