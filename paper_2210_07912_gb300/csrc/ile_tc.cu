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
// Every wait on an mbarrier is bounded; on expiry the kernel raises ILE_FLAG_TIMEOUT, waits once
// more (bounded) for its MMAs, releases its TMEM and returns.
#include <cuda_bf16.h>

#include "ile_internal.cuh"

namespace {

constexpr int TILE = 128;     // samples per CTA = MMA M = TMEM lanes
constexpr int NWMAX = 256;    // max MMA N (columns per window)
constexpr int JCH = 128;      // window bins per chunk
constexpr uint32_t TMEM_COLS = 256;
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

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

template <bool BF16>
__device__ __forceinline__ uint32_t idesc(int n) {
    return (1u << 4) | (Tc<BF16>::FMT << 7) | (Tc<BF16>::FMT << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(TILE >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    if constexpr (BF16) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(id), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(id), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; also gives up early once any CTA of the launch has raised ILE_FLAG_TIMEOUT.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, const unsigned *flags) {
    for (int i = 0; i < WAIT_SPINS; i++) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 1023) == 1023 && (*(volatile const unsigned *)flags & ILE_FLAG_TIMEOUT)) return false;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// hi + lo split of one value; returns the two 16- or 32-bit patterns.
template <bool BF16>
__device__ __forceinline__ void split(float x, uint32_t &hi, uint32_t &lo) {
    if constexpr (BF16) {
        __nv_bfloat16 h = __float2bfloat16_rn(x);
        __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        hi = (uint32_t)__bfloat16_as_ushort(h);
        lo = (uint32_t)__bfloat16_as_ushort(l);
    } else {
        hi = to_tf32(x);
        lo = to_tf32(x - __uint_as_float(hi));
    }
}

// Pack EPC split values of one 16-byte chunk.
template <bool BF16>
__device__ __forceinline__ void pack_chunk(const float *v, uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
    if constexpr (BF16) {
#pragma unroll
        for (int w = 0; w < 4; w++) {
            uint32_t h0, l0, h1, l1;
            split<true>(v[2 * w], h0, l0);
            split<true>(v[2 * w + 1], h1, l1);
            h[w] = h0 | (h1 << 16);
            l[w] = l0 | (l1 << 16);
        }
    } else {
#pragma unroll
        for (int w = 0; w < 4; w++) split<false>(v[w], h[w], l[w]);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

struct TcSmem {
    uint64_t bar;
    uint32_t tmem_base;
    int lohi[2][ILE_MAX_DET];
    int i0[ILE_MAX_DET][TILE];
    float w[ILE_MAX_DET][TILE];
};

template <bool BF16>
__global__ void __launch_bounds__(TILE, 1) ile_tc_kernel(const __grid_constant__ PointParams pp,
                                                        const uint4 *__restrict__ Qhi, const uint4 *__restrict__ Qlo,
                                                        int TP, int KP, IleScratch s, const int *__restrict__ perm,
                                                        int64_t N, double *__restrict__ out, int full_grid,
                                                        unsigned *flags) {
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

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int k = 0; k < K; k++) {
        const int64_t q = valid ? p : p0;
        sm.i0[k][t] = s.I0[(int64_t)k * N + q];
        sm.w[k][t] = valid ? s.W[(int64_t)k * N + q] : 0.f;
    }
    if (t < 2 * ILE_MAX_DET) sm.lohi[t / ILE_MAX_DET][t % ILE_MAX_DET] = (t < ILE_MAX_DET) ? 0x7fffffff : -0x7fffffff;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    for (int k = 0; k < K; k++) {
        int v = sm.i0[k][t];
        int lo = v, hi = v;
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

    const float A = valid ? s.A[p] : 0.f;
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
                    const int r = kc * EPC + e;
                    v[e] = (valid && r < R) ? s.C[((int64_t)k * R + r) * N + p] : 0.f;
                }
                uint4 h, l;
                pack_chunk<BF16>(v, h, l);
                Ahi[kc * TILE + t] = h;
                Alo[kc * TILE + t] = l;
            }
            const int i0 = sm.i0[k][t];
            const float w = sm.w[k][t];
            const int col_lo = sm.lohi[0][k] + j0;
            const int col_hi = sm.lohi[1][k] + j0 + Jc;  // last column used (inclusive)
            for (int wbeg = col_lo; wbeg <= col_hi && !timed_out; wbeg += NWMAX) {
                const int nw = min(NWMAX, col_hi - wbeg + 1);
                const int nwr = (nw + 15) & ~15;
                const uint4 *qh = Qhi + (int64_t)k * KC * TP + wbeg;
                const uint4 *ql = Qlo + (int64_t)k * KC * TP + wbeg;
                for (int i = t; i < KC * nwr; i += TILE) {
                    const int kc = i / nwr, c = i - kc * nwr;
                    Bhi[kc * nwr + c] = qh[(int64_t)kc * TP + c];
                    Blo[kc * nwr + c] = ql[(int64_t)kc * TP + c];
                }
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
                if (t == 0) {
                    tc_fence_after();
                    const uint32_t id = idesc<BF16>(nwr);
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
                            mma<BF16>(tmem, ad, bd, id, acc);
                            acc = 1;
                        }
                    }
                    mma_commit(&sm.bar);
                }
                bool ok = mbar_wait(&sm.bar, phase, flags);
                phase ^= 1u;
                if (__syncthreads_or(!ok)) {
                    timed_out = true;
                    if (t == 0) atomicOr(flags, ILE_FLAG_TIMEOUT);
                    mbar_wait(&sm.bar, phase ^ 1u, flags);
                    break;
                }
                tc_fence_after();
                for (int cb = 0; cb < nwr; cb += 32) {
                    uint32_t r[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)cb, r);
                    const int jbase = wbeg + cb - i0 - j0;  // window bin whose first lerp term is column cb
#pragma unroll
                    for (int q = 0; q < 32; q++) {
                        const float g = __uint_as_float(r[q]);
                        const int jq = jbase + q;
                        if (jq >= 0 && jq < Jc) Dt[jq * TILE + t] += (1.f - w) * g;
                        if (jq >= 1 && jq <= Jc) Dt[(jq - 1) * TILE + t] += w * g;
                    }
                }
                tc_fence_before();
            }
        }
        if (timed_out) break;
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
    if (valid && !full_grid && !timed_out)
        out[perm ? perm[p] : p] = (double)m_run + (double)logf(s_run) - (double)A - (double)pp.log_nt;

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// Split the FP32 data rows Qp [K][R][T] into hi/lo operand rows [K][KC][TP] (16-byte chunks of
// EPC consecutive K-elements r), zero-padded in r up to KP and in t up to TP.
template <bool BF16>
__global__ void split_q_kernel(const float *__restrict__ Qp, int K, int R, int T, int KP, int TP, uint4 *__restrict__ hi,
                               uint4 *__restrict__ lo) {
    constexpr int EPC = Tc<BF16>::EPC;
    const int KC = KP / EPC;
    const int64_t total = (int64_t)K * KC * TP;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int tt = (int)(i % TP);
        const int kc = (int)((i / TP) % KC);
        const int k = (int)(i / ((int64_t)TP * KC));
        float v[EPC];
#pragma unroll
        for (int e = 0; e < EPC; e++) {
            const int r = kc * EPC + e;
            v[e] = (r < R && tt < T) ? Qp[((int64_t)k * R + r) * T + tt] : 0.f;
        }
        uint4 h, l;
        pack_chunk<BF16>(v, h, l);
        hi[i] = h;
        lo[i] = l;
    }
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

int ile_tc_tpad(int T_ext) { return T_ext + NWMAX + 16; }

size_t ile_tc_q_bytes(int prec, int K, int M, int T_ext) {
    const int KP = ile_tc_kpad(prec, M);
    const int KC = KP / (prec == ILE_PREC_BF16X3 ? 8 : 4);
    return (size_t)K * KC * ile_tc_tpad(T_ext) * 16;
}

cudaError_t ile_launch_tc_split(int prec, const PointParams &pp, const float *Qp, void *hi, void *lo, cudaStream_t st) {
    const int KP = ile_tc_kpad(prec, pp.M), TP = ile_tc_tpad(pp.T_ext);
    if (prec == ILE_PREC_BF16X3)
        split_q_kernel<true><<<256, 256, 0, st>>>(Qp, pp.K, 2 * pp.M, pp.T_ext, KP, TP, (uint4 *)hi, (uint4 *)lo);
    else
        split_q_kernel<false><<<256, 256, 0, st>>>(Qp, pp.K, 2 * pp.M, pp.T_ext, KP, TP, (uint4 *)hi, (uint4 *)lo);
    return cudaGetLastError();
}

cudaError_t ile_launch_tc(int prec, const PointParams &pp, const void *hi, const void *lo, IleScratch s,
                          const int *perm, int64_t N, double *out, int full_grid, unsigned *flags, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const int KP = ile_tc_kpad(prec, pp.M), TP = ile_tc_tpad(pp.T_ext);
    const unsigned blocks = (unsigned)((N + TILE - 1) / TILE);
    if (prec == ILE_PREC_BF16X3) {
        const size_t sm = tc_smem_bytes<true>(KP);
        cudaError_t e = cudaFuncSetAttribute(ile_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        ile_tc_kernel<true><<<blocks, TILE, sm, st>>>(pp, (const uint4 *)hi, (const uint4 *)lo, TP, KP, s, perm, N, out,
                                                     full_grid, flags);
    } else {
        const size_t sm = tc_smem_bytes<false>(KP);
        cudaError_t e = cudaFuncSetAttribute(ile_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        ile_tc_kernel<false><<<blocks, TILE, sm, st>>>(pp, (const uint4 *)hi, (const uint4 *)lo, TP, KP, s, perm, N,
                                                      out, full_grid, flags);
    }
    return cudaGetLastError();
}
