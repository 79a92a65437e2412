// ile_plain.cu -- "plain" FP32 CUDA-core path of stages S3 (shifted data term) and S5 (time
// marginalisation).
//
// The data term of Eq. (eq:loglikelihood) at window bin j is
//   D(n, j) = sum_k [ (1 - w_k) G_k(n, i_k + j) + w_k G_k(n, i_k + j + 1) ],
//   G_k(n, t) = sum_r C_k(r, n) Qp_k(r, t)      (r over Re and Im rows: Re(conj(c) Q)),
// where i_k(n) + w_k(n) is the sample's fractional window start in detector k.  One CTA of 256
// threads takes 64 delay-sorted samples, four threads per sample, each thread 16 bins of every
// 64-bin chunk of the window held in registers.  Per (chunk, detector) the tile's columns are
// covered by blocks of 80 (overlapping by the lerp partner): an FP32 register-blocked GEMM (a
// 4-sample x 5-column micro-tile per thread, K = 2M) forms G for the block in shared memory and
// every thread adds the interpolation of its own shifted columns.  After the last detector of a
// chunk each thread folds its bins into a running log-sum-exp; the four threads of a sample merge
// theirs and assemble
//   lnL_t = max_j D + ln sum_j exp(D - max) - A - ln N_t
// in FP64.  The Q columns of the next block are copied asynchronously while the current one is
// contracted.  ~91 KB of shared memory per CTA: two CTAs (16 warps) per SM.
#include "ile_internal.cuh"

namespace {

constexpr int NS = 64;                     // samples per CTA (4 threads each)
constexpr int NT = 256;
constexpr int JW = 64;                     // window bins per chunk
constexpr int JG = 16;                     // bins per thread per chunk
constexpr int WC = 80;                     // columns of one GEMM block (16 column groups x 5)
constexpr int WSTEP = WC - 1;              // blocks overlap by one column: the lerp partner
constexpr int RMAX = 2 * ILE_MAX_MODES;    // real rows of the contraction
constexpr int GROW = WC + 4;               // G row stride (floats)
constexpr int NFILL = (NT / WC) * WC;      // threads that stage the Q block: 240, column tid % WC

// Per-detector value held in registers (selects instead of a dynamically indexed local array).
struct PerDet {
    float v0, v1, v2, v3;
    __device__ float operator()(int k) const { return k == 0 ? v0 : k == 1 ? v1 : k == 2 ? v2 : v3; }
};
struct PerDetI {
    int v0, v1, v2, v3;
    __device__ int operator()(int k) const { return k == 0 ? v0 : k == 1 ? v1 : k == 2 ? v2 : v3; }
};

// Asynchronous 4-byte global -> shared copy (zero-filled when `in` is false; src stays a valid
// address either way), and its group commit / wait.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool in) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(in ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// One CTA: NS samples (processing order n0 .. n0 + NS - 1).  Thread t serves sample t / 4 and the
// bins 16 (t % 4) .. 16 (t % 4) + 15 of every 64-bin chunk, accumulating D in registers.  Per
// (chunk, detector) the tile's column range [min i0 + j0, max i0 + j0 + Jc] is covered by blocks of
// WC columns: a register-blocked FP32 GEMM G = C^T Qp (each thread a 4-sample x 5-column
// micro-tile, K = 2M) into shared memory, then each thread adds the lerp of its own shifted
// columns.  After the last detector of a chunk the thread folds its bins into a running
// log-sum-exp; the four threads of a sample merge theirs at the end and lnL_t is assembled in FP64.
__global__ void __launch_bounds__(NT, 2) ile_plain_kernel(const __grid_constant__ PointParams pp,
                                                          const float *__restrict__ Qp, IleScratch s,
                                                          const int *__restrict__ perm, int64_t N,
                                                          double *__restrict__ out, int full_grid, LoudList loud) {
    extern __shared__ __align__(16) float smem[];
    const int K = pp.K, Nt = pp.Nt, R = 2 * pp.M, T = pp.T_ext;
    float *Cs = smem;                          // [K][RMAX][NS]
    float *Qs = Cs + ILE_MAX_DET * RMAX * NS;  // [2][RMAX][WC]: the block in use and the next one
    float *Gs = Qs + 2 * RMAX * WC;            // [NS][GROW]
    __shared__ int rng[2][8][ILE_MAX_DET];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = tid >> 2, g = tid & 3, jbeg = g * JG;
    const int64_t n0 = (int64_t)blockIdx.x * NS;
    const int ns = (int)min((int64_t)NS, N - n0);
    const bool valid = n < ns;
    const int64_t p = n0 + (valid ? n : 0);  // invalid rows repeat the tile's first sample

    // the tile's coefficients, and this sample's window placement per detector
    for (int i = tid; i < K * R * NS; i += NT) {
        const int nn = i % NS, kr = i / NS;
        Cs[kr / R * RMAX * NS + (kr % R) * NS + nn] = nn < ns ? s.C[(int64_t)kr * N + n0 + nn] : 0.f;
    }
    int i0[ILE_MAX_DET];
    float wt[ILE_MAX_DET];
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        i0[k] = k < K ? s.I0[(int64_t)k * N + p] : 0;
        wt[k] = k < K ? s.W[(int64_t)k * N + p] : 0.f;
    }
    const PerDetI i0d{i0[0], i0[1], i0[2], i0[3]};
    const PerDet wtd{wt[0], wt[1], wt[2], wt[3]};
    // per-detector range of window starts over the tile
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        int lo = i0[k], hi = i0[k];
        for (int o = 16; o; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            rng[0][warp][k] = lo;
            rng[1][warp][k] = hi;
        }
    }
    __syncthreads();
    int tlo[ILE_MAX_DET], thi[ILE_MAX_DET];
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        tlo[k] = rng[0][0][k];
        thi[k] = rng[1][0][k];
#pragma unroll
        for (int w = 1; w < NT / 32; w++) {
            tlo[k] = min(tlo[k], rng[0][w][k]);
            thi[k] = max(thi[k], rng[1][w][k]);
        }
    }
    const PerDetI tlod{tlo[0], tlo[1], tlo[2], tlo[3]}, thid{thi[0], thi[1], thi[2], thi[3]};
    const float A = s.A[p];
    DmargSample dq{};
    if (pp.dm.on) dq = ile_dmarg_sample(pp.dm, A);

    float D[JG];
#pragma unroll
    for (int jj = 0; jj < JG; jj++) D[jj] = 0.f;
    float m_run = -INFINITY, s_run = 0.f;
    // GEMM micro-tile: samples 4 ty .. 4 ty + 3, columns 4 tx .. 4 tx + 3 and 64 + tx
    const int ty = tid >> 4, tx = tid & 15;
    const int fc = tid % WC, fr0 = tid / WC;  // Q staging: column fc, rows fr0, fr0 + NT / WC, ...

    // The blocks in order: chunk j0, detector k, first column cb (steps of WSTEP up to the last column
    // whose lerp pair starts in the chunk).  Block b's Q columns are copied asynchronously into
    // buffer b & 1 while block b - 1 is contracted.
    auto next_block = [&](int &j0, int &k, int &cb) {
        cb += WSTEP;
        if (cb > thid(k) + j0 + min(JW, Nt - j0) - 1) {
            if (++k == K) {
                k = 0;
                j0 += JW;
            }
            cb = tlod(k) + j0;
        }
    };
    auto stage = [&](int buf, int k, int cb) {
        if (tid < NFILL) {
            const int col = cb + fc;
            const bool in = col >= 0 && col < T;
            const float *src = Qp + ((int64_t)k * R + fr0) * T + (in ? col : 0);
            float *dst = Qs + buf * RMAX * WC + fr0 * WC + fc;
            for (int r = fr0; r < R; r += NT / WC) {
                cp_async4(dst, src, in);
                src += (NT / WC) * (int64_t)T;
                dst += (NT / WC) * WC;
            }
        }
        cp_async_commit();
    };
    int j0 = 0, k = 0, cb = tlod(0), buf = 0;
    stage(0, 0, cb);
    while (j0 < Nt) {
        int nj0 = j0, nk = k, ncb = cb;
        next_block(nj0, nk, ncb);
        if (nj0 < Nt)
            stage(buf ^ 1, nk, ncb);  // buffer buf ^ 1 was last read by block b - 1's GEMM, before its G barrier
        else
            cp_async_commit();  // an empty group keeps "all but the newest group" meaning block b
        cp_async_wait_prev();
        __syncthreads();  // block b's columns are in; every thread is done with block b - 1's G
        const int Jc = min(JW, Nt - j0);
        {
            const float *Ck = Cs + k * RMAX * NS;
            const float *Qb = Qs + buf * RMAX * WC;
            // accumulators in sample pairs (4 ty, 4 ty + 1) and (4 ty + 2, 4 ty + 3): one packed FP32
            // FMA (two IEEE fmas, the same results as two fmaf) per pair and column
            float2 acc[2][5];
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int b = 0; b < 5; b++) acc[h][b] = make_float2(0.f, 0.f);
#pragma unroll 6
            for (int r = 0; r < R; r++) {
                const float4 av = *reinterpret_cast<const float4 *>(Ck + r * NS + 4 * ty);
                const float4 b4 = *reinterpret_cast<const float4 *>(Qb + r * WC + 4 * tx);
                const float bv[5] = {b4.x, b4.y, b4.z, b4.w, Qb[r * WC + 64 + tx]};
                const float2 a01 = make_float2(av.x, av.y), a23 = make_float2(av.z, av.w);
#pragma unroll
                for (int b = 0; b < 5; b++) {
                    const float2 bb = make_float2(bv[b], bv[b]);
                    acc[0][b] = ile_f2op_fma(a01, bb, acc[0][b]);
                    acc[1][b] = ile_f2op_fma(a23, bb, acc[1][b]);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                float *g0 = Gs + (4 * ty + 2 * h) * GROW, *g1 = g0 + GROW;
                *reinterpret_cast<float4 *>(g0 + 4 * tx) = make_float4(acc[h][0].x, acc[h][1].x, acc[h][2].x, acc[h][3].x);
                *reinterpret_cast<float4 *>(g1 + 4 * tx) = make_float4(acc[h][0].y, acc[h][1].y, acc[h][2].y, acc[h][3].y);
                g0[64 + tx] = acc[h][4].x;
                g1[64 + tx] = acc[h][4].y;
            }
        }
        __syncthreads();
        {
            // my bins j0 + jbeg + jj read columns c = i0 + j0 + jbeg + jj and c + 1 of the block
            // (each column read once: the partner of bin jj is the first column of bin jj + 1)
            const float w = wtd(k), omw = 1.f - w;
            const float *gr = Gs + n * GROW;
            const int c0 = i0d(k) + j0 + jbeg - cb;
            if (c0 >= 0 && c0 + JG <= WSTEP && jbeg + JG <= Jc) {
                // the usual case: all my bins and their partners lie in this block
                const float *src = gr + c0;
                float vprev = src[0];
#pragma unroll
                for (int jj = 0; jj < JG; jj++) {
                    const float v = src[jj + 1];
                    D[jj] = fmaf(omw, vprev, fmaf(w, v, D[jj]));
                    vprev = v;
                }
            } else {
                float vprev = (c0 >= 0 && c0 < WC) ? gr[c0] : 0.f;
#pragma unroll
                for (int jj = 0; jj < JG; jj++) {
                    const int c = c0 + jj;
                    const float v = (c + 1 >= 0 && c + 1 < WC) ? gr[c + 1] : 0.f;
                    if (jbeg + jj < Jc && c >= 0 && c < WSTEP) D[jj] = fmaf(omw, vprev, fmaf(w, v, D[jj]));
                    vprev = v;
                }
            }
        }
        const int bj0 = j0;  // this block's chunk
        j0 = nj0;
        k = nk;
        cb = ncb;
        buf ^= 1;
        if (j0 == bj0) continue;
        // chunk bj0 complete
        if (pp.dm.on) {
            // ln F(D_j, A) of the chunk's bins: one Chebyshev interpolant per sample through 12 table
            // values (3 per thread; the sample's four threads are consecutive lanes), or per-bin
            // table reads where the sample's data terms span more than ILE_DM_WMAX
            float lo = INFINITY, hi = -INFINITY;
#pragma unroll
            for (int jj = 0; jj < JG; jj++)
                if (jbeg + jj < Jc) {
                    lo = fminf(lo, D[jj]);
                    hi = fmaxf(hi, D[jj]);
                }
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, 1));
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, 2));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, 1));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, 2));
            const DmRange rg = ile_dm_range(lo, hi);
            float fv[3];
#pragma unroll
            for (int i = 0; i < 3; i++)  // thread g: nodes g, g + 4, g + 8
                fv[i] = rg.fit && g + 4 * i < ILE_DM_NODES ? ile_dmarg_lnF(pp.dm, dq, ile_dm_node(rg, g + 4 * i)) : 0.f;
            float f[ILE_DM_NODES];
#pragma unroll
            for (int q = 0; q < ILE_DM_NODES; q++) f[q] = __shfl_sync(0xffffffffu, fv[q / 4], (lane & ~3) | (q % 4));
            if (rg.fit) {
                float c[ILE_DM_NODES];
                ile_dm_coeffs(f, c);
                if (jbeg + JG <= Jc) {
#pragma unroll
                    for (int jj = 0; jj < JG; jj += 2) {
                        const float2 v = ile_dm_eval2(c, rg, make_float2(D[jj], D[jj + 1]));
                        D[jj] = v.x;
                        D[jj + 1] = v.y;
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < JG; jj++)
                        if (jbeg + jj < Jc) D[jj] = ile_dm_eval(c, rg, D[jj]);
                }
            } else {
#pragma unroll
                for (int jj = 0; jj < JG; jj++)
                    if (jbeg + jj < Jc) D[jj] = ile_dmarg_lnF(pp.dm, dq, D[jj]);
            }
        }
        if (full_grid) {
            if (valid) {
                const double An = pp.dm.on ? 0.0 : (double)A;
                const int64_t o = (int64_t)(perm ? perm[p] : p) * Nt + bj0 + jbeg;
#pragma unroll
                for (int jj = 0; jj < JG; jj++)
                    if (jbeg + jj < Jc) out[o + jj] = (double)D[jj] - An;
            }
        } else if (jbeg < Jc) {
            float mc = -INFINITY;
#pragma unroll
            for (int jj = 0; jj < JG; jj++)
                if (jbeg + jj < Jc) mc = fmaxf(mc, D[jj]);
            if (mc > m_run) {
                s_run *= expf(m_run - mc);
                m_run = mc;
            }
#pragma unroll
            for (int jj = 0; jj < JG; jj++)
                if (jbeg + jj < Jc) s_run += expf(D[jj] - m_run);
        }
#pragma unroll
        for (int jj = 0; jj < JG; jj++) D[jj] = 0.f;
    }
    if (full_grid) return;
    // S5: merge the four threads of the sample (consecutive lanes), FP64 assembly
    float m = m_run;
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    float sm = s_run > 0.f ? s_run * expf(m_run - m) : 0.f;
    sm += __shfl_xor_sync(0xffffffffu, sm, 1);
    sm += __shfl_xor_sync(0xffffffffu, sm, 2);
    if (g == 0 && valid) {
        const double An = pp.dm.on ? 0.0 : (double)A;
        const int64_t dst = perm ? perm[p] : p;
        out[dst] = (double)m + (double)logf(sm) - An - (double)pp.log_nt;
        // a sample too loud for FP32 goes to the FP64 refinement (ile_refine.cu)
        if (loud.list && fabsf(m) + A > loud.thr) ile_loud_append(loud, (int)dst);
    }
}

size_t plain_smem() { return sizeof(float) * ((size_t)ILE_MAX_DET * RMAX * NS + 2 * RMAX * WC + (size_t)NS * GROW); }

}  // namespace

cudaError_t ile_launch_plain(const PointParams &pp, const float *Qp, IleScratch s, const int *perm, int64_t N,
                             double *out, int full_grid, LoudList loud, unsigned *flags, cudaStream_t st) {
    (void)flags;
    if (N <= 0) return cudaSuccess;
    if (full_grid || pp.dm.on) loud.list = nullptr;
    const size_t smem = plain_smem();
    cudaError_t e = cudaFuncSetAttribute(ile_plain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (N + NS - 1) / NS;
    ile_plain_kernel<<<(unsigned)blocks, NT, smem, st>>>(pp, Qp, s, perm, N, out, full_grid, loud);
    return cudaGetLastError();
}
