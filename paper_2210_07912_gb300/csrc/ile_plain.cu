// ile_plain.cu -- "plain" FP32 CUDA-core path of stages S3 (shifted data term) and S5 (time
// marginalisation).
//
// The data term of Eq. (eq:loglikelihood) at window bin j is
//   D(n, j) = sum_k [ (1 - w_k) G_k(n, i_k + j) + w_k G_k(n, i_k + j + 1) ],
//   G_k(n, t) = sum_r C_k(r, n) Qp_k(r, t)      (r over Re and Im rows: Re(conj(c) Q)),
// where i_k(n) + w_k(n) is the sample's fractional window start in detector k.  One CTA takes a
// tile of NS samples; for every detector it sweeps the columns the tile needs in chunks of 64:
// an FP32 register-blocked GEMM (each thread a (NS/16) x 4 micro-tile) forms G for the chunk in
// shared memory, and a gather adds each sample's interpolated, shifted row into its window
// accumulator D (shared memory, one row of N_t per sample).  After the last detector one warp
// per sample takes the log-sum-exp over the window (S5) and assembles
//   lnL_t = max_j D + ln sum_j exp(D - max) - A - ln N_t
// in FP64.
#include "ile_internal.cuh"

namespace {

constexpr int TCOL = 64;                   // columns per chunk
constexpr int RMAX = 2 * ILE_MAX_MODES;    // real rows of the contraction

template <int NS>
__global__ void __launch_bounds__(256) ile_plain_kernel(const __grid_constant__ PointParams pp,
                                                        const float *__restrict__ Qp, IleScratch s,
                                                        const int *__restrict__ perm, int64_t N,
                                                        double *__restrict__ out, int full_grid, LoudList loud) {
    constexpr int RS = NS / 16;  // samples per thread in the micro-tile
    extern __shared__ float smem[];
    const int Nt = pp.Nt, R = 2 * pp.M, T = pp.T_ext;
    float *Ds = smem;                   // [NS][Nt]
    float *Cs = Ds + NS * Nt;           // [RMAX][NS]
    float *Qs = Cs + RMAX * NS;         // [RMAX][TCOL]
    float *Gs = Qs + RMAX * TCOL;       // [NS][TCOL + 1]
    __shared__ int i0s[NS];
    __shared__ float ws[NS];
    __shared__ int red[2][8];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n0 = (int64_t)blockIdx.x * NS;
    const int ns = (int)min((int64_t)NS, N - n0);

    for (int i = tid; i < NS * Nt; i += 256) Ds[i] = 0.f;

    for (int k = 0; k < pp.K; k++) {
        __syncthreads();
        if (tid < NS) {
            int nn = tid < ns ? tid : 0;
            i0s[tid] = s.I0[(int64_t)k * N + n0 + nn];
            ws[tid] = s.W[(int64_t)k * N + n0 + nn];
        }
        for (int i = tid; i < R * NS; i += 256) {
            int r = i / NS, nn = i - r * NS;
            Cs[r * NS + nn] = nn < ns ? s.C[((int64_t)k * R + r) * N + n0 + nn] : 0.f;
        }
        __syncthreads();
        // column range needed by the tile: [min i0, max i0 + Nt]
        int lo = 0x7fffffff, hi = -0x7fffffff;
        for (int i = tid; i < ns; i += 256) {
            lo = min(lo, i0s[i]);
            hi = max(hi, i0s[i]);
        }
        for (int o = 16; o; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            red[0][warp] = lo;
            red[1][warp] = hi;
        }
        __syncthreads();
        lo = red[0][0];
        hi = red[1][0];
        for (int w = 1; w < 8; w++) {
            lo = min(lo, red[0][w]);
            hi = max(hi, red[1][w]);
        }
        const int cend = hi + Nt;  // last column used (inclusive)

        for (int c0 = lo; c0 <= cend; c0 += TCOL) {
            __syncthreads();
            for (int i = tid; i < R * TCOL; i += 256) {
                int r = i / TCOL, c = i - r * TCOL;
                int col = c0 + c;
                Qs[r * TCOL + c] = (col >= 0 && col < T) ? Qp[((int64_t)k * R + r) * T + col] : 0.f;
            }
            __syncthreads();
            {
                const int ty = tid >> 4, tx = tid & 15;
                float acc[RS][4];
#pragma unroll
                for (int i = 0; i < RS; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = 0.f;
                for (int r = 0; r < R; r++) {
                    float a[RS];
#pragma unroll
                    for (int i = 0; i < RS; i++) a[i] = Cs[r * NS + ty * RS + i];
                    float4 b = *reinterpret_cast<const float4 *>(&Qs[r * TCOL + tx * 4]);
#pragma unroll
                    for (int i = 0; i < RS; i++) {
                        acc[i][0] = fmaf(a[i], b.x, acc[i][0]);
                        acc[i][1] = fmaf(a[i], b.y, acc[i][1]);
                        acc[i][2] = fmaf(a[i], b.z, acc[i][2]);
                        acc[i][3] = fmaf(a[i], b.w, acc[i][3]);
                    }
                }
#pragma unroll
                for (int i = 0; i < RS; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) Gs[(ty * RS + i) * (TCOL + 1) + tx * 4 + j] = acc[i][j];
            }
            __syncthreads();
            // gather: window bin j of sample n takes columns i0 + j (weight 1 - w) and i0 + j + 1 (weight w)
            for (int nn = warp; nn < ns; nn += 8) {
                const int i0 = i0s[nn];
                const float wt = ws[nn];
                const int jlo = max(0, c0 - 1 - i0), jhi = min(Nt - 1, c0 + TCOL - 1 - i0);
                const float *g = Gs + nn * (TCOL + 1);
                float *d = Ds + nn * Nt;
                for (int j = jlo + lane; j <= jhi; j += 32) {
                    int c = i0 + j - c0;
                    float v = 0.f;
                    if (c >= 0) v = (1.f - wt) * g[c];
                    if (c + 1 < TCOL) v = fmaf(wt, g[c + 1], v);
                    d[j] += v;
                }
            }
        }
    }
    __syncthreads();

    // S5: log-sum-exp over the window, FP64 assembly (distance-marginalised: ln F(D_j, A) per bin)
    const double log_nt = log((double)Nt);
    for (int nn = warp; nn < ns; nn += 8) {
        float *d = Ds + nn * Nt;
        double A = (double)s.A[n0 + nn];
        const int64_t dst = perm ? (int64_t)perm[n0 + nn] : n0 + nn;
        if (pp.dm.on) {
            const DmargSample q = ile_dmarg_sample(pp.dm, (float)A);
            for (int j = lane; j < Nt; j += 32) d[j] = ile_dmarg_lnF(pp.dm, q, d[j]);
            A = 0.0;
        }
        if (full_grid) {
            for (int j = lane; j < Nt; j += 32) out[dst * Nt + j] = (double)d[j] - A;
            continue;
        }
        float m = -INFINITY;
        for (int j = lane; j < Nt; j += 32) m = fmaxf(m, d[j]);
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        float sum = 0.f;
        for (int j = lane; j < Nt; j += 32) sum += expf(d[j] - m);
        for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) {
            out[dst] = (double)m + (double)logf(sum) - A - log_nt;
            // a sample too loud for FP32 goes to the FP64 refinement (ile_refine.cu)
            if (loud.list && fabsf(m) + (float)A > loud.thr) ile_loud_append(loud, (int)dst);
        }
    }
}

template <int NS>
size_t plain_smem(const PointParams &pp) {
    return sizeof(float) * ((size_t)NS * pp.Nt + RMAX * NS + RMAX * TCOL + (size_t)NS * (TCOL + 1));
}

template <int NS>
cudaError_t launch(const PointParams &pp, const float *Qp, IleScratch s, const int *perm, int64_t N, double *out,
                   int full_grid, LoudList loud, cudaStream_t st) {
    size_t smem = plain_smem<NS>(pp);
    cudaError_t e = cudaFuncSetAttribute(ile_plain_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (N + NS - 1) / NS;
    ile_plain_kernel<NS><<<(unsigned)blocks, 256, smem, st>>>(pp, Qp, s, perm, N, out, full_grid, loud);
    return cudaGetLastError();
}

}  // namespace

cudaError_t ile_launch_plain(const PointParams &pp, const float *Qp, IleScratch s, const int *perm, int64_t N,
                             double *out, int full_grid, LoudList loud, unsigned *flags, cudaStream_t st) {
    (void)flags;
    if (N <= 0) return cudaSuccess;
    if (full_grid || pp.dm.on) loud.list = nullptr;
    if (pp.Nt <= 512) return launch<64>(pp, Qp, s, perm, N, out, full_grid, loud, st);
    return launch<32>(pp, Qp, s, perm, N, out, full_grid, loud, st);
}
