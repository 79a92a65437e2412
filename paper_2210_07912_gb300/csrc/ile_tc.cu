// ile_tc.cu -- split-precision tensor-core path of stages S3 (shifted data term) and S5 (time
// marginalisation) on sm_103a: tcgen05.mma with operands in shared memory and the FP32
// accumulator in tensor memory (TMEM).
//
// For one tile of 128 samples (sorted by delay, so their window starts are close) and one
// detector k, the data term needs G_k(n, t) = sum_r C_k(n, r) Qp_k(r, t) over the columns
// [min_n i0 + j0, max_n i0 + j0 + J] of a window chunk j0 .. j0 + J.  That is a dense GEMM with
// M = 128 samples, N = the column window (<= 256 per MMA), K = 2M real rows padded to KP.  Both
// operands are split into hi + lo parts (BF16 for kind::f16, TF32 for kind::tf32) and the MMA
// accumulates hi*hi + hi*lo + lo*hi in FP32 (the lo*lo term is dropped).  Thread t of the CTA
// owns TMEM lane t = sample t: it reads its accumulator row with tcgen05.ld and adds
// (1 - w) G(i0 + j) + w G(i0 + j + 1) into its private column of the window accumulator D in
// shared memory; after the last detector of a chunk it folds the chunk into a running
// log-sum-exp.  lnL_t = m + ln s - A - ln N_t is assembled in FP64.
//
// Shared-memory operand layout (no swizzle, K-major canonical layout): a "core matrix" is 8 rows
// x 16 bytes; row n of K-chunk kc sits at byte (kc * rows + n) * 16, so the leading-dimension
// byte offset (between K-chunks) is rows * 16 and the stride-dimension byte offset (between
// 8-row groups) is 128.
//
// This kernel serves the TF32x3 mode (and BF16x3 when the fused kernel of ile_tc2.cu cannot be used).
// Every wait on an mbarrier is bounded; on expiry the kernel raises ILE_FLAG_TIMEOUT, waits once
// more (bounded) for its MMAs, releases its TMEM and returns.
#include "ile_internal.cuh"
#include "ile_tcgen05.cuh"

using namespace ile_tc;

namespace {

constexpr int TILE = 128;     // samples per CTA = MMA M = TMEM lanes
constexpr int NWMAX = 80;     // max MMA N (columns per window)
constexpr int JCH = 64;       // window bins per chunk
constexpr uint32_t TMEM_COLS = 128;  // power of two >= NWMAX rounded up to the 32-column loads
constexpr int TPAD = 256;     // columns of the tiled operand past T_ext (room for any window)
constexpr int WAIT_SPINS = 1 << 20;

template <bool BF16>
struct Tc;
template <>
struct Tc<true> {
    static constexpr int EPC = 8;  // elements per 16-byte chunk
    static constexpr int KS = 16;  // MMA K
    static constexpr uint32_t FMT = 1;  // BF16
};
template <>
struct Tc<false> {
    static constexpr int EPC = 4;
    static constexpr int KS = 8;
    static constexpr uint32_t FMT = 2;  // TF32
};

__device__ __forceinline__ int64_t qtile_index(int k, int kc, int t, int KC, int TP);

struct TcSmem {
    uint64_t bar;
    uint32_t tmem_base;
    int lohi[2][ILE_MAX_DET];
};

// Per-detector value held in registers (selects instead of a dynamically indexed local array).
template <typename T>
struct Det {
    T v0, v1, v2, v3;
    __device__ T operator()(int k) const { return k == 0 ? v0 : k == 1 ? v1 : k == 2 ? v2 : v3; }
};

template <bool BF16>
__global__ void __launch_bounds__(TILE, 2) ile_tc_kernel(const __grid_constant__ PointParams pp,
                                                        const uint4 *__restrict__ Qhi, const uint4 *__restrict__ Qlo,
                                                        int TP, int KP, IleScratch s, const int *__restrict__ perm,
                                                        int64_t N, double *__restrict__ out, int full_grid,
                                                        LoudList loud, unsigned *flags) {
    constexpr int EPC = Tc<BF16>::EPC, KS = Tc<BF16>::KS;
    extern __shared__ __align__(1024) uint8_t dsm[];
    __shared__ TcSmem sm;
    const int KC = KP / EPC;
    uint4 *Ahi = reinterpret_cast<uint4 *>(dsm);
    uint4 *Alo = Ahi + KC * TILE;
    uint4 *Bhi = Alo + KC * TILE;
    uint4 *Blo = Bhi + KC * NWMAX;
    float *Dt = reinterpret_cast<float *>(Blo + KC * NWMAX);  // [JCH][TILE]

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int K = pp.K, R = 2 * pp.M, Nt = pp.Nt;
    const int64_t p = (int64_t)blockIdx.x * TILE + t;
    const bool valid = p < N;
    const int64_t p0 = (int64_t)blockIdx.x * TILE;  // always valid

    if (warp == 0) tmem_alloc(&sm.tmem_base, TMEM_COLS);
    if (t == 0) {
        mbar_init(&sm.bar, 1);
        mbar_init_fence();
    }
    int i0v[ILE_MAX_DET];
    float wv[ILE_MAX_DET];
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        const int64_t q = valid ? p : p0;
        i0v[k] = k < K ? s.I0[(int64_t)k * N + q] : 0;
        wv[k] = (k < K && valid) ? s.W[(int64_t)k * N + q] : 0.f;
    }
    const Det<int> i0d{i0v[0], i0v[1], i0v[2], i0v[3]};
    const Det<float> wd{wv[0], wv[1], wv[2], wv[3]};
    if (t < 2 * ILE_MAX_DET) sm.lohi[t / ILE_MAX_DET][t % ILE_MAX_DET] = (t < ILE_MAX_DET) ? 0x7fffffff : -0x7fffffff;
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem_base;
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        if (k >= K) break;
        int lo = i0v[k], hi = i0v[k];
        for (int o = 16; o; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            atomicMin(&sm.lohi[0][k], lo);
            atomicMax(&sm.lohi[1][k], hi);
        }
    }
    __syncthreads();

    float A = valid ? s.A[p] : 0.f;
    DmargSample dq{};
    if (pp.dm.on) {
        dq = ile_dmarg_sample(pp.dm, A);  // per-bin terms become ln F(D_j, A); nothing is subtracted
        A = 0.f;
    }
    float m_run = -INFINITY, s_run = 0.f;
    uint32_t phase = 0;
    bool timed_out = false;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;

    for (int j0 = 0; j0 < Nt && !timed_out; j0 += JCH) {
        const int Jc = min(JCH, Nt - j0);
        for (int jj = 0; jj < Jc; jj++) Dt[jj * TILE + t] = 0.f;
        for (int k = 0; k < K && !timed_out; k++) {
            // A operand: row t = coefficients of sample t for detector k, split hi/lo
            for (int kc = 0; kc < KC; kc++) {
                float v[EPC];
#pragma unroll
                for (int e = 0; e < EPC; e++) {
                    const int r = kc * EPC + e;  // operand K index 2a + {Re, Im}; C rows are Re then Im
                    const int row = (r & 1) ? R / 2 + r / 2 : r / 2;
                    v[e] = (valid && r < R) ? s.C[((int64_t)k * R + row) * N + p] : 0.f;
                }
                uint4 h, l;
                pack_chunk<BF16>(v, h, l);
                Ahi[kc * TILE + t] = h;
                Alo[kc * TILE + t] = l;
            }
            const int i0 = i0d(k);
            const float w = wd(k);
            const int col_lo = sm.lohi[0][k] + j0;
            const int col_hi = sm.lohi[1][k] + j0 + Jc;  // last column used (inclusive)
            for (int wbeg = col_lo; wbeg <= col_hi && !timed_out; wbeg += NWMAX) {
                const int nw = min(NWMAX, col_hi - wbeg + 1);
                const int nwr = (nw + 15) & ~15;
                for (int i = t; i < KC * nwr; i += TILE) {
                    const int kc = i / nwr, c = i - kc * nwr;
                    const int64_t qi = qtile_index(k, kc, wbeg + c, KC, TP);
                    Bhi[kc * nwr + c] = Qhi[qi];
                    Blo[kc * nwr + c] = Qlo[qi];
                }
                fence_async_smem();
                fence_before();
                __syncthreads();
                if (t == 0) {
                    fence_after();
                    const uint32_t id = idesc(Tc<BF16>::FMT, TILE, nwr);
                    const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo);
                    const uint32_t b_hi = smem_u32(Bhi), b_lo = smem_u32(Blo);
                    const uint32_t a_lbo = TILE * 16, b_lbo = (uint32_t)nwr * 16;
                    const int nks = KP / KS;
                    uint32_t acc = 0;
#pragma unroll 1
                    for (int pass = 0; pass < 3; pass++) {
                        const uint32_t ab = (pass == 2) ? a_lo : a_hi;
                        const uint32_t bb = (pass == 1) ? b_lo : b_hi;
                        for (int ks = 0; ks < nks; ks++) {
                            const uint64_t ad = sdesc(ab + ks * 2 * a_lbo, a_lbo, 128);
                            const uint64_t bd = sdesc(bb + ks * 2 * b_lbo, b_lbo, 128);
                            if constexpr (BF16)
                                mma_bf16(tmem, ad, bd, id, acc);
                            else
                                mma_tf32(tmem, ad, bd, id, acc);
                            acc = 1;
                        }
                    }
                    mma_commit(&sm.bar);
                }
                bool ok = mbar_wait(&sm.bar, phase, flags, ILE_FLAG_TIMEOUT, WAIT_SPINS);
                phase ^= 1u;
                if (__syncthreads_or(!ok)) {
                    timed_out = true;
                    if (t == 0) atomicOr(flags, ILE_FLAG_TIMEOUT);
                    mbar_wait(&sm.bar, phase ^ 1u, flags, 0u, WAIT_SPINS);
                    break;
                }
                fence_after();
                for (int cb = 0; cb < nwr; cb += 32) {
                    uint32_t r[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)cb, r);
                    const int jbase = wbeg + cb - i0 - j0;  // window bin whose first lerp term is column cb
#pragma unroll
                    for (int q = 0; q < 32; q++) {
                        const float g = __uint_as_float(r[q]);
                        const int jq = jbase + q;
                        // columns at or past nw belong to the next window (or lie past the last one)
                        const bool col = cb + q < nw;
                        if (col && jq >= 0 && jq < Jc) Dt[jq * TILE + t] += (1.f - w) * g;
                        if (col && jq >= 1 && jq <= Jc) Dt[(jq - 1) * TILE + t] += w * g;
                    }
                }
                fence_before();
            }
        }
        if (timed_out) break;
        if (pp.dm.on) {
            // ln F(D_j, A) of the chunk's bins: a Chebyshev interpolant through 12 table values, or
            // per-bin table reads where the data terms span more than ILE_DM_WMAX
            float lo = INFINITY, hi = -INFINITY;
            for (int jj = 0; jj < Jc; jj++) {
                lo = fminf(lo, Dt[jj * TILE + t]);
                hi = fmaxf(hi, Dt[jj * TILE + t]);
            }
            const DmRange rg = ile_dm_range(lo, hi);
            if (rg.fit) {
                float f[ILE_DM_NODES], c[ILE_DM_NODES];
#pragma unroll
                for (int k = 0; k < ILE_DM_NODES; k++) f[k] = ile_dmarg_lnF(pp.dm, dq, ile_dm_node(rg, k));
                ile_dm_coeffs(f, c);
                for (int jj = 0; jj < Jc; jj++) Dt[jj * TILE + t] = ile_dm_eval(c, rg, Dt[jj * TILE + t]);
            } else {
                for (int jj = 0; jj < Jc; jj++) Dt[jj * TILE + t] = ile_dmarg_lnF(pp.dm, dq, Dt[jj * TILE + t]);
            }
        }
        if (full_grid) {
            if (valid) {
                const int64_t o = (int64_t)(perm ? perm[p] : p) * Nt + j0;
                for (int jj = 0; jj < Jc; jj++) out[o + jj] = (double)Dt[jj * TILE + t] - (double)A;
            }
            continue;
        }
        float mc = -INFINITY;
        for (int jj = 0; jj < Jc; jj++) mc = fmaxf(mc, Dt[jj * TILE + t]);
        if (mc > m_run) {
            s_run *= expf(m_run - mc);
            m_run = mc;
        }
        for (int jj = 0; jj < Jc; jj++) s_run += expf(Dt[jj * TILE + t] - m_run);
    }
    if (valid && !full_grid && !timed_out) {
        const int64_t dst = perm ? perm[p] : p;
        out[dst] = (double)m_run + (double)logf(s_run) - (double)A - (double)pp.log_nt;
        // a sample too loud for single precision goes to the FP64 refinement (ile_refine.cu)
        if (loud.list && fabsf(m_run) + A > loud.thr) ile_loud_append(loud, (int)dst);
    }

    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// Split the FP32 data rows Qp [K][R][T] (Re rows then Im rows) into hi/lo operand rows
// [K][KC][TP]: 16-byte chunks of EPC consecutive operand K indices r = 2a + {0: Re, 1: Im},
// zero-padded in r up to KP and in t up to TP.
// Split the FP32 data rows Qp [K][R][T] (Re rows then Im rows) into hi/lo operand chunks:
// 16-byte chunks of EPC consecutive operand K indices r = 2a + {0: Re, 1: Im} (zero-padded up
// to KP), stored core-matrix tiled as [K][TP/8][KC][8 columns] so that a window of 8-aligned
// columns is one contiguous block (zero-padded in t up to TP).
template <bool BF16>
__global__ void split_q_kernel(const float *__restrict__ Qp, int K, int R, int T, int KP, int TP, uint4 *__restrict__ hi,
                               uint4 *__restrict__ lo) {
    constexpr int EPC = Tc<BF16>::EPC;
    const int KC = KP / EPC;
    const int64_t total = (int64_t)K * KC * TP;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int t8 = (int)(i % 8);
        const int kc = (int)((i / 8) % KC);
        const int64_t grp = i / (8 * KC);  // k * TP/8 + t / 8
        const int k = (int)(grp / (TP / 8));
        const int tt = (int)(grp % (TP / 8)) * 8 + t8;
        float v[EPC];
#pragma unroll
        for (int e = 0; e < EPC; e++) {
            const int r = kc * EPC + e;
            const int row = (r & 1) ? R / 2 + r / 2 : r / 2;
            v[e] = (r < R && tt < T) ? Qp[((int64_t)k * R + row) * T + tt] : 0.f;
        }
        uint4 h, l;
        pack_chunk<BF16>(v, h, l);
        hi[i] = h;
        lo[i] = l;
    }
}

// The quadratic-term block (real form of U_k, V_k; rows r = 2a + {Re, Im}, row stride KPq of the
// host array, four 32-column blocks) into columns TP - ILE_QCOLS .. TP - ILE_QCOLS + ILE_QUAD_NCOL
// of the tiled split layout, its blocks packed to ILE_QUAD_NCOL / 4 columns.
template <bool BF16>
__global__ void split_quad_kernel(const float *__restrict__ quad, int K, int KPq, int KP, int TP,
                                  uint4 *__restrict__ hi, uint4 *__restrict__ lo) {
    constexpr int EPC = Tc<BF16>::EPC;
    constexpr int NCOL = ILE_QUAD_NCOL, BLK = NCOL / 4;
    const int KC = KP / EPC;
    const int64_t total = (int64_t)K * KC * NCOL;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)(i % NCOL);
        const int kc = (int)((i / NCOL) % KC);
        const int k = (int)(i / ((int64_t)NCOL * KC));
        const int src = (col / BLK) * (ILE_QCOLS / 4) + col % BLK;
        float v[EPC];
#pragma unroll
        for (int e = 0; e < EPC; e++) {
            const int r = kc * EPC + e;
            v[e] = r < KPq ? quad[((int64_t)k * KPq + r) * ILE_QCOLS + src] : 0.f;
        }
        uint4 h, l;
        pack_chunk<BF16>(v, h, l);
        const int t = TP - ILE_QCOLS + col;
        const int64_t o = (((int64_t)k * (TP / 8) + t / 8) * KC + kc) * 8 + (t & 7);
        hi[o] = h;
        lo[o] = l;
    }
}

// Index (in 16-byte chunks) of K-chunk kc of column t of detector k in the tiled split layout.
__device__ __forceinline__ int64_t qtile_index(int k, int kc, int t, int KC, int TP) {
    return (((int64_t)k * (TP / 8) + t / 8) * KC + kc) * 8 + (t & 7);
}

template <bool BF16>
size_t tc_smem_bytes(int KP) {
    const int KC = KP / Tc<BF16>::EPC;
    return (size_t)16 * (2 * KC * TILE + 2 * KC * NWMAX) + sizeof(float) * JCH * TILE;
}

}  // namespace

int ile_tc_kpad(int prec, int M) {
    const int R = 2 * M;
    return prec == ILE_PREC_BF16X3 ? (R + 15) & ~15 : (R + 7) & ~7;
}

// Time columns of the tiled operand: T_ext plus room for a full window past the end, then the
// ILE_QCOLS quadratic-term columns (used by the BF16X3 fused kernel) at column tpad - ILE_QCOLS.
int ile_tc_tpad(int T_ext) { return ((T_ext + TPAD + 16 + 7) & ~7) + ILE_QCOLS; }

size_t ile_tc_q_bytes(int prec, int K, int M, int T_ext) {
    const int KP = ile_tc_kpad(prec, M);
    const int KC = KP / (prec == ILE_PREC_BF16X3 ? 8 : 4);
    return (size_t)K * KC * ile_tc_tpad(T_ext) * 16;
}

namespace {
// FP32 operand rows of Q from its FP64 copy: Qp[k][a][t] = Re Q, Qp[k][M + a][t] = Im Q; a
// non-finite entry raises ILE_FLAG_NONFINITE in *chk.
__global__ void q_convert_kernel(const double2 *__restrict__ Q64, int K, int M, int T, float *__restrict__ Qp,
                                 unsigned *__restrict__ chk) {
    const int64_t total = (int64_t)K * M * T;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 q = Q64[i];
        const int64_t ka = i / T;
        const int t = (int)(i - ka * T), k = (int)(ka / M), a = (int)(ka - (int64_t)k * M);
        Qp[((int64_t)k * 2 * M + a) * T + t] = (float)q.x;
        Qp[((int64_t)k * 2 * M + M + a) * T + t] = (float)q.y;
        bad = bad || !isfinite(q.x) || !isfinite(q.y);
    }
    if (bad) atomicOr(chk, ILE_FLAG_NONFINITE);
}
}  // namespace

cudaError_t ile_launch_q_convert(const double2 *Q64, int K, int M, int T, float *Qp, unsigned *chk, cudaStream_t st) {
    q_convert_kernel<<<256, 256, 0, st>>>(Q64, K, M, T, Qp, chk);
    return cudaGetLastError();
}

cudaError_t ile_launch_tc_split(int prec, const PointParams &pp, const float *Qp, const float *quad, void *hi,
                                void *lo, cudaStream_t st) {
    const int KP = ile_tc_kpad(prec, pp.M), TP = ile_tc_tpad(pp.T_ext);
    // the host's real-form array has BF16 operand rows (KP rounded up to 16)
    const int KPq = ile_tc_kpad(ILE_PREC_BF16X3, pp.M);
    if (prec == ILE_PREC_BF16X3) {
        split_q_kernel<true><<<256, 256, 0, st>>>(Qp, pp.K, 2 * pp.M, pp.T_ext, KP, TP, (uint4 *)hi, (uint4 *)lo);
        if (quad) split_quad_kernel<true><<<64, 256, 0, st>>>(quad, pp.K, KPq, KP, TP, (uint4 *)hi, (uint4 *)lo);
    } else {
        split_q_kernel<false><<<256, 256, 0, st>>>(Qp, pp.K, 2 * pp.M, pp.T_ext, KP, TP, (uint4 *)hi, (uint4 *)lo);
        if (quad) split_quad_kernel<false><<<64, 256, 0, st>>>(quad, pp.K, KPq, KP, TP, (uint4 *)hi, (uint4 *)lo);
    }
    return cudaGetLastError();
}

cudaError_t ile_launch_tc(int prec, const PointParams &pp, const void *hi, const void *lo, IleScratch s,
                          const int *perm, int64_t N, double *out, int full_grid, LoudList loud, unsigned *flags,
                          cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    if (full_grid || pp.dm.on) loud.list = nullptr;
    const int KP = ile_tc_kpad(prec, pp.M), TP = ile_tc_tpad(pp.T_ext);
    const unsigned blocks = (unsigned)((N + TILE - 1) / TILE);
    if (prec == ILE_PREC_BF16X3) {
        const size_t sm = tc_smem_bytes<true>(KP);
        cudaError_t e = cudaFuncSetAttribute(ile_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        ile_tc_kernel<true><<<blocks, TILE, sm, st>>>(pp, (const uint4 *)hi, (const uint4 *)lo, TP, KP, s, perm, N, out,
                                                     full_grid, loud, flags);
    } else {
        const size_t sm = tc_smem_bytes<false>(KP);
        cudaError_t e = cudaFuncSetAttribute(ile_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        ile_tc_kernel<false><<<blocks, TILE, sm, st>>>(pp, (const uint4 *)hi, (const uint4 *)lo, TP, KP, s, perm, N,
                                                      out, full_grid, loud, flags);
    }
    return cudaGetLastError();
}
