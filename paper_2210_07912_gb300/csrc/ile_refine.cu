// ile_refine.cu -- FP64 refinement of loud samples (S1-S5 recomputed for the samples whose
// likelihood terms are too large for single precision).
//
// The log-space assembly lnL_t = max_j D + ln sum_j e^{D_j - max} - A - ln N_t (Eq.
// (eq:loglikelihood) with the time marginalisation of the subsection "Choices for finite-precision
// floating point arithmetic and overflow") keeps every intermediate finite, but the absolute error
// of a single-precision data term D or quadratic term A grows with their size: about 1e-6 of
// |D| + A for the split-precision tensor-core products and 3e-7 for FP32 arithmetic (geometry,
// coefficients and window placement are FP32 in every fast path).  For SNRs of tens (App. "Choices
// for finite-precision floating point arithmetic and overflow" discusses rho ~ 35 and beyond) that
// exceeds 1e-3.  The fast kernels therefore append every sample with |max_j D| + A above a
// per-precision threshold to a device list, and this kernel recomputes those samples, one warp per
// sample:
//   * geometry (wave frame, antenna factors, delays, window placement), harmonics, coefficients
//     c_klm = (D_ref/D) F_k Y_lm and the quadratic term A = 1/4 sum_k [c^H U c + Re(c^T V c)] in FP64
//     from FP64 copies of the detector data, U and V;
//   * the data term of every window bin in FP32 from the FP64 window placement;
//   * in FP64 the data term of every bin that matters and is large (D_j >= max_j D - 30 and
//     |D_j| > threshold: the bins within e^-30 of the peak carry the log-sum-exp);
//   * the log-sum-exp of the bins in FP64 (exponentials of FP64 differences in FP32).
// The result replaces the fast path's lnL_t of the sample.  Nothing else is read from the fast
// path, so the refined value does not depend on the precision that flagged it.
#include "ile_internal.cuh"

namespace {

constexpr int RF_WARPS = 8;
constexpr double RF_C = 299792458.0;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One listed sample n of one point (the whole warp): lnL_t recomputed into out[n].
__device__ void refine_one(const Refine64 &P, const double2 *__restrict__ Q64, const double2 *__restrict__ U64,
                           const double2 *__restrict__ V64, const float *__restrict__ Qp,
                           const double *__restrict__ samples, int64_t N, int64_t n, double *__restrict__ out,
                           unsigned *flags, float (*csh)[2 * ILE_MAX_MODES]) {
    const int lane = threadIdx.x & 31;
    const int K = P.K, M = P.M, Nt = P.Nt, T = P.T_ext;
    double th[ILE_NDIM];
#pragma unroll
    for (int d = 0; d < ILE_NDIM; d++) th[d] = samples[(int64_t)d * N + n];
    // ---- S1 in FP64: wave frame (X x Y = -n), antenna factors F = F+ + i Fx, delays
    double sg, cg, sd, cd, sp, cp;
    sincos(P.gmst - th[0], &sg, &cg);
    sincos(th[1], &sd, &cd);
    sincos(th[2], &sp, &cp);
    const double X[3] = {-cp * sg - sp * cg * sd, -cp * cg + sp * sg * sd, sp * cd};
    const double Y[3] = {sp * sg - cp * cg * sd, sp * cg + cp * sg * sd, cp * cd};
    const double nv[3] = {cd * cg, -cd * sg, sd};
    // lane k < K: detector k's antenna factors and window start
    double Fr = 0, Fi = 0, x0 = 0;
    if (lane < K) {
        const double *Dm = P.det_tensor[lane];
        double DX[3], DY[3];
        for (int a = 0; a < 3; a++) {
            DX[a] = Dm[3 * a] * X[0] + Dm[3 * a + 1] * X[1] + Dm[3 * a + 2] * X[2];
            DY[a] = Dm[3 * a] * Y[0] + Dm[3 * a + 1] * Y[1] + Dm[3 * a + 2] * Y[2];
        }
        Fr = (X[0] * DX[0] + X[1] * DX[1] + X[2] * DX[2]) - (Y[0] * DY[0] + Y[1] * DY[1] + Y[2] * DY[2]);
        Fi = (X[0] * DY[0] + X[1] * DY[1] + X[2] * DY[2]) + (Y[0] * DX[0] + Y[1] * DX[1] + Y[2] * DX[2]);
        const double dt = -(P.det_pos[lane][0] * nv[0] + P.det_pos[lane][1] * nv[1] + P.det_pos[lane][2] * nv[2]) / RF_C;
        x0 = (th[6] + dt - P.t_start) * P.fs - 0.5 * Nt;
    }
    double Frk[ILE_MAX_DET], Fik[ILE_MAX_DET], wk[ILE_MAX_DET];
    int ik[ILE_MAX_DET];
    bool in_range = true;
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        Frk[k] = __shfl_sync(0xffffffffu, Fr, k);
        Fik[k] = __shfl_sync(0xffffffffu, Fi, k);
        const double xs = __shfl_sync(0xffffffffu, x0, k);
        const double xk = P.nearest ? rint(xs) : xs;  // nearest-sample mode: weight 0 at the rounded start
        const double fl = floor(xk);
        ik[k] = k < K ? (int)fl : 0;
        wk[k] = xk - fl;
        if (k < K) in_range = in_range && fl >= 0.0 && fl + Nt <= (double)(T - 1);
    }
    bool finite = th[5] > 0.0;
#pragma unroll
    for (int d = 0; d < ILE_NDIM; d++) finite = finite && isfinite(th[d]);
    if (!finite || !in_range) {
        // the fast path has flagged the sample (non-finite / range); keep its placeholder
        if (lane == 0 && finite && !in_range) atomicOr(flags, ILE_FLAG_RANGE);
        return;
    }
    // ---- S2 in FP64: lane a < M holds Y_a and the coefficients c_ka = (D_ref/D) F_k Y_a
    const double scale = P.d_ref / th[5];
    double cr[ILE_MAX_DET] = {0, 0, 0, 0}, ci[ILE_MAX_DET] = {0, 0, 0, 0};
    if (lane < M) {
        double sh, ch;
        sincos(0.5 * th[3], &sh, &ch);
        double cpw[9], spw[9];  // powers of cos(iota/2), sin(iota/2)
        cpw[0] = spw[0] = 1.0;
        for (int e = 1; e < 9; e++) {
            cpw[e] = cpw[e - 1] * ch;
            spw[e] = spw[e - 1] * sh;
        }
        const Mode64 &md = P.mode[lane];
        double amp = 0.0;
        for (int t = 0; t < md.nterms; t++) amp += md.coef[t] * cpw[md.p[t]] * spw[md.q[t]];
        amp *= md.norm;
        double sm, cm;
        sincos((double)md.m * th[4], &sm, &cm);
        const double yr = amp * cm, yi = amp * sm;
#pragma unroll
        for (int k = 0; k < ILE_MAX_DET; k++) {
            if (k < K) {
                cr[k] = scale * (Frk[k] * yr - Fik[k] * yi);
                ci[k] = scale * (Frk[k] * yi + Fik[k] * yr);
                csh[k][lane] = (float)cr[k];
                csh[k][M + lane] = (float)ci[k];
            }
        }
    }
    __syncwarp();
    // ---- S4 in FP64: lane a forms row a of U_k c_k and V_k c_k
    double aq = 0.0;
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        if (k >= K) break;
        double zr = 0, zi = 0, wr = 0, wi = 0;
        for (int b = 0; b < M; b++) {
            const double br = __shfl_sync(0xffffffffu, cr[k], b), bi = __shfl_sync(0xffffffffu, ci[k], b);
            if (lane < M) {
                const double2 u = U64[((size_t)k * M + lane) * M + b], v = V64[((size_t)k * M + lane) * M + b];
                zr += u.x * br - u.y * bi;
                zi += u.x * bi + u.y * br;
                wr += v.x * br - v.y * bi;
                wi += v.x * bi + v.y * br;
            }
        }
        // Re(conj(c_a) z_a) + Re(c_a w_a)
        if (lane < M) aq += (cr[k] * zr + ci[k] * zi) + (cr[k] * wr - ci[k] * wi);
    }
    const double A = 0.25 * warp_sum(aq);
    // ---- S3 in FP32 for every bin: lane l takes the 16-bin blocks j0 = 16 l, 16 l + 512, ...
    constexpr int JB = 16;
    const int nblk = (Nt + 32 * JB - 1) / (32 * JB);  // blocks per lane (1 for N_t <= 512)
    float D[2][JB];
    float mloc = -INFINITY;
    for (int bq = 0; bq < 2; bq++) {
        const int j0 = (bq * 32 + lane) * JB;
#pragma unroll
        for (int jj = 0; jj < JB; jj++) D[bq][jj] = 0.f;
        if (bq >= nblk || j0 >= Nt) continue;
#pragma unroll
        for (int k = 0; k < ILE_MAX_DET; k++) {
            if (k >= K) break;
            const float w = (float)wk[k], omw = 1.f - w;
            float G[JB + 1];
#pragma unroll
            for (int t = 0; t <= JB; t++) G[t] = 0.f;
            const int c0 = ik[k] + j0;
            const int tmax = min(JB, T - 1 - c0);  // columns c0 .. c0 + tmax stay inside the series
            for (int r = 0; r < 2 * M; r++) {
                const float c = csh[k][r];
                const float *q = Qp + ((size_t)k * 2 * M + r) * T + c0;
#pragma unroll
                for (int t = 0; t <= JB; t++)
                    if (t <= tmax) G[t] = fmaf(c, __ldg(q + t), G[t]);
            }
#pragma unroll
            for (int jj = 0; jj < JB; jj++) D[bq][jj] = fmaf(omw, G[jj], fmaf(w, G[jj + 1], D[bq][jj]));
        }
#pragma unroll
        for (int jj = 0; jj < JB; jj++)
            if (j0 + jj < Nt) mloc = fmaxf(mloc, D[bq][jj]);
    }
    const float m32 = warp_maxf(mloc);
    // every bin from here on is an offset from m32 (exact for the bins near the peak, whose
    // FP32 values are within a factor 2 of it; a relative 6e-8 of at most ~30 otherwise)
    for (int bq = 0; bq < nblk; bq++)
#pragma unroll
        for (int jj = 0; jj < JB; jj++) D[bq][jj] -= m32;
    // ---- S3 in FP64 for the bins that carry the log-sum-exp and are large: the warp computes
    // one bin at a time (lane a adds mode a of every detector), the owning lane keeps it
    for (int bq = 0; bq < nblk; bq++) {
#pragma unroll 1
        for (int jj = 0; jj < JB; jj++) {
            const int j = (bq * 32 + lane) * JB + jj;
            const float off = D[bq][jj];
            unsigned mask = __ballot_sync(0xffffffffu, j < Nt && off >= -30.f && fabsf(off + m32) > P.thr);
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const int jt = (bq * 32 + src) * JB + jj;
                double part = 0.0;
                if (lane < M) {
#pragma unroll
                    for (int k = 0; k < ILE_MAX_DET; k++) {
                        if (k >= K) break;
                        const double2 *q = Q64 + ((size_t)k * M + lane) * T + ik[k] + jt;
                        const double2 q0 = q[0], q1 = q[1];
                        const double qr = (1.0 - wk[k]) * q0.x + wk[k] * q1.x;
                        const double qi = (1.0 - wk[k]) * q0.y + wk[k] * q1.y;
                        part += cr[k] * qr + ci[k] * qi;  // Re(conj(c) Q)
                    }
                }
                const double d64 = warp_sum(part);
                if (lane == src) D[bq][jj] = (float)(d64 - (double)m32);
            }
        }
    }
    // ---- S5: log-sum-exp over the bins relative to their maximum, FP64 assembly
    float mo = -INFINITY;
    for (int bq = 0; bq < nblk; bq++)
#pragma unroll
        for (int jj = 0; jj < JB; jj++)
            if ((bq * 32 + lane) * JB + jj < Nt) mo = fmaxf(mo, D[bq][jj]);
    mo = warp_maxf(mo);
    float sl = 0.f;
    for (int bq = 0; bq < nblk; bq++)
#pragma unroll
        for (int jj = 0; jj < JB; jj++)
            if ((bq * 32 + lane) * JB + jj < Nt) sl += expf(D[bq][jj] - mo);
    const double ssum = warp_sum((double)sl);
    if (lane == 0) out[n] = (double)m32 + (double)mo + log(ssum) - A - P.log_nt;
}

// Single point: list[0] = count, list[1 + 2 i] = point (0), list[2 + 2 i] = caller index.
__global__ void __launch_bounds__(32 * RF_WARPS) refine_kernel(const __grid_constant__ Refine64 P,
                                                               const double2 *__restrict__ Q64,
                                                               const double2 *__restrict__ U64,
                                                               const double2 *__restrict__ V64,
                                                               const float *__restrict__ Qp,
                                                               const double *__restrict__ samples, int64_t N,
                                                               const int *__restrict__ list, int64_t cap,
                                                               double *__restrict__ out, unsigned *flags) {
    __shared__ float csh[RF_WARPS][ILE_MAX_DET][2 * ILE_MAX_MODES];  // FP32 coefficients: Re rows, then Im
    const int warp = threadIdx.x >> 5;
    const int count = (int)min((int64_t)list[0], cap);
    for (int i = blockIdx.x * RF_WARPS + warp; i < count; i += gridDim.x * RF_WARPS)
        refine_one(P, Q64, U64, V64, Qp, samples, N, list[2 + 2 * i], out, flags, csh[warp]);
}

// Batched run: list[1 + 2 i] = point, list[2 + 2 i] = the sample's index within the point.
__global__ void __launch_bounds__(32 * RF_WARPS) brefine_kernel(const RefinePoint *__restrict__ pts,
                                                                const int *__restrict__ list, int64_t cap,
                                                                unsigned *flags) {
    __shared__ float csh[RF_WARPS][ILE_MAX_DET][2 * ILE_MAX_MODES];
    const int warp = threadIdx.x >> 5;
    const int count = (int)min((int64_t)list[0], cap);
    for (int i = blockIdx.x * RF_WARPS + warp; i < count; i += gridDim.x * RF_WARPS) {
        const RefinePoint &q = pts[list[1 + 2 * i]];
        refine_one(q.r, q.Q64, q.U64, q.V64, q.Qp, q.samples, q.N, list[2 + 2 * i], q.out, flags, csh[warp]);
    }
}

}  // namespace

cudaError_t ile_launch_refine(const Refine64 &P, const double2 *Q64, const double2 *U64, const double2 *V64,
                              const float *Qp, const double *samples, int64_t N, const int *list, int64_t cap,
                              double *out, unsigned *flags, int n_sm, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const int64_t need = (N + RF_WARPS - 1) / RF_WARPS;
    const unsigned grid = (unsigned)(need < 4 * n_sm ? need : 4 * n_sm);
    refine_kernel<<<grid, 32 * RF_WARPS, 0, st>>>(P, Q64, U64, V64, Qp, samples, N, list, cap, out, flags);
    return cudaGetLastError();
}

cudaError_t ile_launch_batch_refine(const RefinePoint *pts, int64_t n_total, const int *list, int64_t cap,
                                    unsigned *flags, int n_sm, cudaStream_t st) {
    if (n_total <= 0) return cudaSuccess;
    const int64_t need = (n_total + RF_WARPS - 1) / RF_WARPS;
    const unsigned grid = (unsigned)(need < 4 * n_sm ? need : 4 * n_sm);
    brefine_kernel<<<grid, 32 * RF_WARPS, 0, st>>>(pts, list, cap, flags);
    return cudaGetLastError();
}
