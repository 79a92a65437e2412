// ile_prep.cu -- per-sample stages S1 (geometry), S2 (mode coefficients) and S4 (quadratic term).
//
// One thread per extrinsic sample, in processing order (optionally a permutation of the caller's
// order; the per-sample outputs are written at the processing position).  For each detector k it forms the antenna factor
// F_k = F+ + i Fx, the window start x0_k = (t_c + dt_k - t_start) f_s - N_t/2 (split into an
// integer index and a lerp weight), and the coefficients c_klm = (D_ref/D) F_k Y_lm
// (Eq. (eq:loglikelihood), first line).  The quadratic term
//   A = 1/4 (D_ref/D)^2 sum_k [ |F_k|^2 y^H U_k y + Re(F_k^2 y^T V_k y) ]      (second line)
// uses the pair products conj(y_a) y_b and y_a y_b once for all detectors, with U and V staged
// in shared memory as upper-triangle pairs and the harmonics in a per-thread column of a shared
// table.  Everything is FP32; the result feeds the FP64
// per-sample assembly of the contraction kernels.
#include "ile_internal.cuh"

namespace {

constexpr int PREP_NT = 256;

__global__ void __launch_bounds__(PREP_NT) ile_prep_kernel(const __grid_constant__ PointParams pp,
                                                       const float4 *__restrict__ UV,
                                                       const double *__restrict__ samples,
                                                       const int *__restrict__ perm, int64_t N, IleScratch s,
                                                       unsigned *flags) {
    extern __shared__ float4 uv_s[];  // [K][P], then the y table
    const int M = pp.M, K = pp.K, P = M * (M + 1) / 2;
    for (int i = threadIdx.x; i < K * P; i += blockDim.x) uv_s[i] = UV[i];
    __syncthreads();
    // n: position in the (sorted) processing order; src: the sample's index in the caller's arrays
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int64_t src = perm ? (int64_t)perm[n] : n;

    double th[ILE_NDIM];
    bool finite = true;
#pragma unroll
    for (int d = 0; d < ILE_NDIM; d++) {
        th[d] = samples[(int64_t)d * N + src];
        finite = finite && isfinite(th[d]);
    }
    if (!finite || th[5] <= 0.0) {
        atomicOr(flags, ILE_FLAG_NONFINITE);
        th[0] = th[1] = th[2] = th[3] = th[4] = th[6] = 0.0;
        th[5] = 1.0;
    }
    const float ra = (float)th[0], dec = (float)th[1], psi = (float)th[2];
    const float iota = (float)th[3], phi = (float)th[4], tc = (float)th[6];
    // distance-marginalised mode: coefficients and quadratic term at D = D_ref
    const float scale = pp.dm.on ? 1.f : pp.d_ref / (float)th[5];

    float Fr[ILE_MAX_DET], Fi[ILE_MAX_DET], x0[ILE_MAX_DET];
    ile_sample_geometry(pp, ra, dec, psi, tc, Fr, Fi, x0);
    // every interpolation pair (i0 + j, i0 + j + 1), j < N_t, must lie inside [0, T_ext - 1]
    bool in_range = true;
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        if (k >= K) break;
        float fl = floorf(x0[k]);
        in_range = in_range && (fl >= 0.f) && (fl + (float)pp.Nt <= (float)(pp.T_ext - 1));
    }
    if (!in_range) atomicOr(flags, ILE_FLAG_RANGE);
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        if (k >= K) break;
        float fl = floorf(x0[k]);
        // a flagged sample gets a harmless in-range placement so that no kernel loops over a
        // runaway column range; the call reports ILE_E_RANGE and its result is not used
        s.I0[(int64_t)k * N + n] = in_range ? (int)fl : 0;
        s.W[(int64_t)k * N + n] = in_range ? x0[k] - fl : 0.f;
    }

    // harmonics with every power at a compile-time index (registers) and e^{i m phi} from powers of
    // e^{i phi}, into this thread's column of the shared y table: the mode and pair loops below stay
    // rolled (fully unrolled, they overflow the instruction cache)
    float2 *ys = reinterpret_cast<float2 *>(uv_s + K * P);  // [M][PREP_NT]
    {
        float cpow[9], spow[9], er[5], ei[5];
        ile_half_angle_powers(iota, cpow, spow);
        ile_phase_powers(phi, er, ei);
#pragma unroll 1
        for (int a = 0; a < M; a++) {
            float yr, yi;
            ile_sylm_fast(pp.mode[a], cpow, spow, er, ei, yr, yi);
            ys[a * PREP_NT + threadIdx.x] = make_float2(yr, yi);
        }
    }
    const int R = 2 * M;
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        if (k >= K) break;
        const float fr = scale * Fr[k], fi = scale * Fi[k];
        float *Ck = s.C + (int64_t)k * R * N + n;
#pragma unroll 1
        for (int a = 0; a < M; a++) {
            const float2 y = ys[a * PREP_NT + threadIdx.x];
            Ck[(int64_t)a * N] = fr * y.x - fi * y.y;
            Ck[(int64_t)(M + a) * N] = fr * y.y + fi * y.x;
        }
    }

    float au[ILE_MAX_DET] = {0.f, 0.f, 0.f, 0.f}, avr[ILE_MAX_DET] = {0.f, 0.f, 0.f, 0.f},
          avi[ILE_MAX_DET] = {0.f, 0.f, 0.f, 0.f};
    int p = 0;
#pragma unroll 1
    for (int a = 0; a < M; a++) {
        const float2 ya = ys[a * PREP_NT + threadIdx.x];
#pragma unroll 1
        for (int b = a; b < M; b++, p++) {
            const float2 yb = ys[b * PREP_NT + threadIdx.x];
            const float qr = ya.x * yb.x + ya.y * yb.y, qi = ya.x * yb.y - ya.y * yb.x;  // conj(y_a) y_b
            const float pr = ya.x * yb.x - ya.y * yb.y, pi = ya.x * yb.y + ya.y * yb.x;  // y_a y_b
#pragma unroll
            for (int k = 0; k < ILE_MAX_DET; k++) {
                if (k < K) {
                    const float4 u = uv_s[k * P + p];
                    au[k] += u.x * qr - u.y * qi;
                    avr[k] += u.z * pr - u.w * pi;
                    avi[k] += u.z * pi + u.w * pr;
                }
            }
        }
    }
    float A = 0.f;
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        if (k >= K) break;
        float f2 = Fr[k] * Fr[k] + Fi[k] * Fi[k];
        float g_r = Fr[k] * Fr[k] - Fi[k] * Fi[k], g_i = 2.f * Fr[k] * Fi[k];  // F^2
        A += f2 * au[k] + (g_r * avr[k] - g_i * avi[k]);
    }
    s.A[n] = 0.25f * scale * scale * A;
}

}  // namespace

cudaError_t ile_launch_prep(const PointParams &pp, const float *UV, const double *samples, const int *perm, int64_t N,
                            IleScratch s, unsigned *flags, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const int P = pp.M * (pp.M + 1) / 2;
    const size_t smem = sizeof(float4) * pp.K * P + sizeof(float2) * pp.M * PREP_NT;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(ile_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (N + PREP_NT - 1) / PREP_NT;
    ile_prep_kernel<<<(unsigned)blocks, PREP_NT, smem, st>>>(pp, (const float4 *)UV, samples, perm, N, s, flags);
    return cudaGetLastError();
}
