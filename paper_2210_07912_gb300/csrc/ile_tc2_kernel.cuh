// ile_tc2_kernel.cuh -- the fused, pipelined split-precision tensor-core kernel for stages S1-S5 on
// sm_103a, shared by the BF16x3 launchers (ile_tc2.cu, single point and batch) and the TF32x3
// launcher (ile_tc3.cu, single point).
//
// One persistent CTA per SM walks 128-sample tiles of the delay-sorted samples.  19 warps:
//
//   16 math warps: warp w serves TMEM lane quadrant q = w % 4 (samples 32q .. 32q+31 of the
//   tile) and bin group g = w / 4, so each sample has four threads (g = 0..3):
//     * S1/S2: the four threads of a sample read its geometry (F_k, window start i0_k + w_k,
//       staged by the prefetch warp) and form a quarter of the harmonics Y_lm each (compile-time
//       powers per (l, m)); the four threads share the K x KC chunks of the sample's coefficients
//       c_klm = (D_ref/D) F_k Y_lm, split hi/lo and written as the MMA A operand (K index
//       2a + {Re, Im} of mode a, as in the split Q rows): BF16 pairs in shared memory for BF16x3,
//       TF32 values in the sample's own TMEM lane (tcgen05.st) for TF32x3;
//     * S4: per detector, MMA jobs against the real form of U_k and V_k leave U_k c and V_k c in
//       TMEM; thread g dots its 32-column block with the coefficients, and the four shares give
//       A(n) = 1/4 sum_k [c_k^H U_k c_k + Re(c_k^T V_k c_k)];
//     * S3/S5 epilogue for every data job: load the sample's accumulator columns from TMEM, keep
//       the 17 it needs (bins 16g .. 16g+15 and the lerp partner) in a thread-private strip of
//       shared memory, and add (1 - w) G(i0 + j) + w G(i0 + j + 1) into its window accumulator
//       D[16] (registers); after the last detector of a chunk, fold D into a running
//       log-sum-exp.  At the end of a tile the four threads' (max, sum) pairs are merged in FP64.
//   warp 17, lane 0 (copy warp): for every job (chunk of 64 window bins x detector x column
//   window of <= 120 columns) bulk-copy the Q window (hi and lo rows, one contiguous block each)
//   into a ring of NB shared buffers as soon as a slot is free;
//   warp 16, lane 0 (MMA warp): issue 3 x KP/16 tcgen05.mma kind::f16 (BF16x3) or 3 x KP/8
//   kind::tf32 with the A operand read from TMEM (TF32x3) per job (hi*hi + hi*lo + lo*hi, FP32
//   accumulation) into one of the TMEM accumulator buffers (three of 128 columns for BF16x3; two
//   beside the 2 K KP columns of the A operand for TF32x3);
//   warp 18 (prefetch warp): gathers the next tile's sample parameters through the sort
//   permutation and computes their geometry (S1) into shared memory while the current tile is in
//   flight.
//
// Hand-offs are mbarriers: bfull/bempty (B ring), tfull/tempty (TMEM buffers), aready (A operand
// and the tile's column ranges written; waited on by all roles), tdone (per-thread log-sum-exp
// partials written), sready (geometry staged; the prefetch warp refills the stage once yready
// shows that every math thread has read it).  The copy and math warps enumerate the jobs
// identically (the quadratic-term jobs, copied before the tile is ready, then (chunk, detector,
// window)); the copy warp publishes each job's detector and width with its B slot and the MMA
// warp follows that sequence.  A tile whose column spread does not fit one window is covered by
// overlapping windows, each sample reading the single window that holds all the columns it needs;
// when every detector fits one window the math warps take a shorter job loop.  Every wait is
// bounded; on expiry the kernel raises ILE_FLAG_TIMEOUT (all CTAs then stop waiting), releases its
// TMEM and returns.  A sample's result depends only on its own parameters (each accumulator
// element sums K in a fixed order, and the lerp and log-sum-exp follow the sample's own bins), so
// neither the tile it lands in nor the window widths change it.
#pragma once
#include "ile_internal.cuh"
#include "ile_tcgen05.cuh"

using namespace ile_tc;

namespace {

constexpr int TILE = 128;
constexpr int NGRP = 4;                    // threads per sample
constexpr int NMATH = TILE * NGRP;         // 512 math threads
constexpr int DMC_ROWS = 4 + ILE_DM_NODES;  // per-sample interpolant store (distance marginalisation)
constexpr int MMA_WARP = NMATH / 32;        // warp 16: tcgen05.mma issue
constexpr int COPY_WARP = MMA_WARP + 1;    // warp 17: bulk copies of the Q windows
constexpr int PREF_WARP = COPY_WARP + 1;   // warp 18: gathers the next tile's sample parameters
constexpr int NTHREADS = NMATH + 96;
constexpr int JW = 64;                     // window bins per chunk
constexpr int JG = JW / NGRP;              // bins per thread per chunk
constexpr int NWIN = 128;                  // columns per TMEM accumulator buffer (= max MMA N here)
constexpr int NWCOL = 120;                 // default window columns (+ up to 7 for 8-column alignment <= NWIN)
constexpr int NWCOL_MIN = JW + 2;          // a window must hold one chunk's columns plus the lerp partner
constexpr int NTB = 3;                     // BF16x3: TMEM accumulator buffers (jobs in flight between MMA and math warps)
constexpr int NTB_TF32 = 2;                // TF32x3: two buffers beside the A operand
constexpr uint32_t TMEM_COLS = 512;        // power of two >= NTB * NWIN
constexpr int NBMAX = 4;                   // B ring depth upper bound
constexpr int SLEEPS = 200000;             // bounded sleeping waits: SLEEPS x SLEEP_NS at most
constexpr uint32_t SLEEP_NS = 10000;
constexpr int RSTRIDE = 34;                // smallest per-thread row: 32 staged columns + 2 spare words
constexpr float ILE_LOG2E_F = 1.4426950408889634f;  // log2(e)

// Operand variants of the kernel: BF16x3 with the A operand in shared memory and three 128-column
// accumulator buffers; BF16x3 with A in TMEM and three 112-column buffers; BF16x3 with A in TMEM
// and two 160-column buffers (wider windows, more shared memory for the B ring: a choice of the
// batch autotuner); TF32x3 with A in TMEM and two 96-column buffers.  A in TMEM: row n of the tile
// in lane n, detector k's hi values then its lo values, KP values each, in consecutive 32-bit
// columns (two BF16 or one TF32 value per column), at most acol_of columns; the accumulator
// buffers follow.
enum : int { OP_BF16_SMEM = 0, OP_BF16_TMEM = 1, OP_TF32_TMEM = 2, OP_BF16_TMEM_W = 3, OP_BF16_SMEM_N = 4 };
// (OP_BF16_SMEM_N: A in shared memory with three 112-column buffers and B slots, which leaves the
// room for 36-word staging rows; the single-point launch)
__host__ __device__ constexpr int acol_of(int op) {
    return op == OP_TF32_TMEM ? 320 : op == OP_BF16_TMEM ? 176 : op == OP_BF16_TMEM_W ? 192 : 0;
}
__host__ __device__ constexpr int ntb_of(int op) { return op == OP_TF32_TMEM || op == OP_BF16_TMEM_W ? 2 : NTB; }
__host__ __device__ constexpr int bw_of(int op) {
    return op == OP_BF16_SMEM ? NWIN
           : op == OP_BF16_SMEM_N ? 112
                                  : ((int)TMEM_COLS - acol_of(op)) / ntb_of(op) / 16 * 16;
}
// Staging-row stride (words): 36 keeps every row 16-byte aligned (a TMEM block is staged with
// four 16-byte stores, conflict-free per quarter warp; 1% faster than 34 on the single-point
// launch); the other variants keep 34 (8-byte stores, half-warp conflict-free), with which the
// batch's largest operands and the TF32x3 variant's fourth B slot fit.
__host__ __device__ constexpr int rstride_of(int op) { return op == OP_BF16_SMEM_N || op == OP_BF16_TMEM ? 36 : RSTRIDE; }
// TMEM columns of a point's A operand (K detectors, KP values per row and part)
__host__ __device__ constexpr int acols_needed(int op, int K, int KP) { return op == OP_TF32_TMEM ? 2 * K * KP : K * KP; }
static_assert(bw_of(OP_TF32_TMEM) == 96 && bw_of(OP_BF16_TMEM) == 112 && bw_of(OP_BF16_TMEM_W) == 160,
              "accumulator buffers");
static_assert(acol_of(OP_BF16_TMEM_W) + 2 * bw_of(OP_BF16_TMEM_W) <= (int)TMEM_COLS, "wide BF16x3 TMEM layout");
static_assert(acol_of(OP_BF16_TMEM) + NTB * bw_of(OP_BF16_TMEM) <= (int)TMEM_COLS, "BF16x3 TMEM layout");
static_assert(acol_of(OP_TF32_TMEM) + NTB_TF32 * bw_of(OP_TF32_TMEM) <= (int)TMEM_COLS, "TF32x3 TMEM layout");
static_assert(ILE_QUAD_NCOL <= 96 && 96 - 7 >= NWCOL_MIN, "a quadratic-term job and a window fit every buffer");

// 2^x with the SFU's base-2 exponential (approximate; flushes subnormal results to zero)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Sm {
    uint64_t bfull[NBMAX], bempty[NBMAX], tfull[NTB], tempty[NTB], yready, aready, s4done, tdone, sready;
    uint64_t dmx[4];  // distance-marginalised chunks: the four warps of a TMEM lane quarter exchange values
    uint32_t tmem_base;
    int wlo[4][ILE_MAX_DET], whi[4][ILE_MAX_DET];
    int2 dkr[NMATH / 32][ILE_MAX_DET];  // per math warp and detector: (min, max) of i0 - tile lo
    uint32_t jinfo[NBMAX];  // job of each B slot for the MMA warp: detector | nwr << 4 | last-of-tile << 16
};

// Register-resident per-detector value (the selects avoid dynamic indexing).
struct Det4 {
    int v0, v1, v2, v3;
    __device__ int operator()(int k) const { return k == 0 ? v0 : k == 1 ? v1 : k == 2 ? v2 : v3; }
};
struct Det4f {
    float v0, v1, v2, v3;
    __device__ float operator()(int k) const { return k == 0 ? v0 : k == 1 ? v1 : k == 2 ? v2 : v3; }
};

// One data-term job of a tile: chunk c (bins j0 .. j0 + Jc), detector k, window w of W.
struct Job {
    int j0, Jc, k, w, W, step, wbeg, wbeg8, nwr;  // window [wbeg8, wbeg8 + nwr), wbeg8 = wbeg rounded down to 8
};

// Enumerates the data-term jobs of a tile from the tile's per-detector column range [lo_k, hi_k]
// of window starts (the tile's quadratic-term jobs come before them and are walked separately).
// The copy and math warps walk the same sequence.
struct JobIter {
    int Nt, K, nwcol;
    Det4 lo, hi;
    int c, k, w;
    bool done;
    __device__ JobIter(int Nt_, int K_, int nwcol_, Det4 lo_, Det4 hi_)
        : Nt(Nt_), K(K_), nwcol(nwcol_), lo(lo_), hi(hi_), c(0), k(0), w(0), done(false) {}
    __device__ Job get() const {
        Job j;
        j.j0 = c * JW;
        j.Jc = min(JW, Nt - j.j0);
        j.k = k;
        j.w = w;
        const int col_lo = lo(k) + j.j0, col_hi = hi(k) + j.j0 + j.Jc;  // inclusive
        const int total = col_hi - col_lo + 1;
        if (total <= nwcol) {
            j.W = 1;
            j.step = nwcol;
        } else {
            j.step = nwcol - j.Jc - 1;
            j.W = 1 + (total - nwcol + j.step - 1) / j.step;
        }
        j.wbeg = col_lo + w * j.step;
        j.wbeg8 = j.wbeg & ~7;
        const int nw = min(nwcol, col_hi - j.wbeg + 1) + (j.wbeg - j.wbeg8);
        j.nwr = (nw + 15) & ~15;
        return j;
    }
    // advance past job j (the job get() returned for the current position)
    __device__ void next_from(const Job &j) {
        if (++w < j.W) return;
        w = 0;
        if (++k < K) return;
        k = 0;
        if ((++c) * JW >= Nt) done = true;
    }
};

// Tile column range of detector k from the per-quadrant partial ranges.
__device__ __forceinline__ void tile_range(const int (*wlo)[ILE_MAX_DET], const int (*whi)[ILE_MAX_DET], int K,
                                           Det4 &lo, Det4 &hi) {
    int l[ILE_MAX_DET], h[ILE_MAX_DET];
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        l[k] = k < K ? min(min(wlo[0][k], wlo[1][k]), min(wlo[2][k], wlo[3][k])) : 0;
        h[k] = k < K ? max(max(whi[0][k], whi[1][k]), max(whi[2][k], whi[3][k])) : 0;
    }
    lo = Det4{l[0], l[1], l[2], l[3]};
    hi = Det4{h[0], h[1], h[2], h[3]};
}

__device__ __forceinline__ bool wait1(uint64_t *bar, uint32_t parity, const unsigned *flags) {
    return mbar_wait_sleep(bar, parity, flags, ILE_FLAG_TIMEOUT, SLEEPS, SLEEP_NS);
}

__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, const unsigned *flags) {
    return __all_sync(0xffffffffu, wait1(bar, parity, flags));
}

// Work item `it` of the launch: one 128-sample tile of one intrinsic point.  A single-point
// launch walks the tiles of `one`; a batched launch walks (point, tile) pairs from `items`.
template <bool BATCH>
__device__ __forceinline__ const Tc2Point &work_item(const Tc2Point &one, const Tc2Point *__restrict__ pts,
                                                     const int2 *__restrict__ items, int64_t it, int64_t &tile) {
    if constexpr (BATCH) {
        const int2 w = items[it];
        tile = w.y;
        return pts[w.x];
    } else {
        tile = it;
        return one;
    }
}

// Shared-memory layout (LK detectors, LKC 16-byte K-chunks: the point's own sizes for a
// single-point launch, the largest of the batch otherwise; BW = NWIN for BF16x3, tf32_bufw for
// TF32x3, whose A operand lives in TMEM instead):
//   A [LK][2][LKC][TILE] (BF16x3 only) | B [NB][2][LKC][BW] | rows [NMATH][RSTRIDE] | aq_s [NMATH]
//   | ls_s [NMATH] | geo [14][TILE]
// A math thread's row holds the two 16-column TMEM blocks its bins need; aq_s and ls_s its share
// of the quadratic term and its partial log-sum-exp; geo the tile's per-sample geometry (antenna
// factors, window starts, iota, phi), computed by the prefetch warp from the parameters it gathers
// through the sort permutation while the previous tile is in flight.  Before
// the job loop the rows area holds the tile's harmonics table y [M][TILE] (float2).
// ADJ: the adjoint's D(n, j) pass (grid mode 2), which also writes each sample's coefficients,
// window placements and quadratic term (Tc2Point::sC, sI0, sW, sA)
template <bool BATCH, bool DM, int OP, bool ADJ = false>
__global__ void __launch_bounds__(NTHREADS, 1)
    ile_tc2_kernel(const __grid_constant__ Tc2Point one, const Tc2Point *__restrict__ pts,
                   const int2 *__restrict__ items, int64_t nitems, int LK, int LKC, int LNP, int NB, int nwcol,
                   int full_grid, unsigned *flags) {
    extern __shared__ __align__(1024) uint8_t dsm[];
    __shared__ Sm sm;
    (void)LNP;
    // operand element layout: 16-byte chunks of 8 BF16 or 4 TF32 values; A in TMEM or shared memory
    constexpr bool TF32 = OP == OP_TF32_TMEM, ATM = OP != OP_BF16_SMEM && OP != OP_BF16_SMEM_N;
    // distance marginalisation keeps each sample's interpolant across chunks (a 15 KB store), except
    // in the variant with A in shared memory, whose four-detector launches have no room for it
    constexpr bool DMREUSE = DM && OP != OP_BF16_SMEM;
    constexpr int RS = rstride_of(OP);  // staging-row stride
    constexpr int EPC = TF32 ? 4 : 8;
    constexpr int NTBv = ntb_of(OP);
    static_assert(NTBv <= NTB, "barrier arrays");
    // quadratic-term job width: the real form of U_k, V_k in four blocks of QN / 4 columns
    constexpr int QN = ILE_QUAD_NCOL;
    constexpr int acol = acol_of(OP);  // first accumulator column
    constexpr int bw = bw_of(OP);      // accumulator buffer and B slot width
    uint4 *A = reinterpret_cast<uint4 *>(dsm);                                        // [K][2][KC][TILE]
    uint4 *B = A + (ATM ? 0 : (size_t)LK * 2 * LKC * TILE);                           // [NB][2][LKC][BW]
    float *rows = reinterpret_cast<float *>(B + (size_t)NB * 2 * LKC * bw);           // [NMATH][RS]
    float *aq_s = rows + RS * NMATH;                                                  // [NMATH]
    float2 *ls_s = reinterpret_cast<float2 *>(aq_s + NMATH);                           // [NMATH]
    float *geo = reinterpret_cast<float *>(ls_s + NMATH);                              // [14][TILE]
    // distance-marginalised mode: each sample's current interpolant, [DMC_ROWS][TILE] (rows: range
    // low and high end, middle, 1 / half-width, the 10 monomial coefficients), and the chunk-range
    // exchange, two buffers of [NMATH]
    float *dmc = geo + 14 * TILE;
    float2 *dmr = reinterpret_cast<float2 *>(dmc + DMC_ROWS * TILE);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == MMA_WARP) tmem_alloc(&sm.tmem_base, TMEM_COLS);
    if (tid == 0) {
        for (int b = 0; b < NBMAX; b++) {
            mbar_init(&sm.bfull[b], 1);
            mbar_init(&sm.bempty[b], 1);
        }
        for (int b = 0; b < NTBv; b++) {
            mbar_init(&sm.tfull[b], 1);
            mbar_init(&sm.tempty[b], NMATH / 32);  // one arrival per math warp
        }
        // the math-warp barriers count one arrival per warp (lane 0, after the warp synchronises)
        mbar_init(&sm.yready, NMATH / 32);
        mbar_init(&sm.aready, NMATH / 32);
        mbar_init(&sm.s4done, NMATH / 32);
        mbar_init(&sm.tdone, NMATH / 32);
        mbar_init(&sm.sready, 32);
        for (int q = 0; q < 4; q++) mbar_init(&sm.dmx[q], NGRP);
        mbar_init_fence();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem_base;
    bool failed = false;

    if (warp == COPY_WARP) {
        // ------------------------------------------------------------------ copy warp
        if (lane == 0) {
            uint32_t gcopy = 0, tiles_done = 0;
            uint32_t bb = 0, bpar = 0;  // ring slot and phase parity of copy gcopy
            for (int64_t it = blockIdx.x; it < nitems && !failed; it += gridDim.x, tiles_done++) {
                int64_t tile;
                const Tc2Point &pt = work_item<BATCH>(one, pts, items, it, tile);
                const int K = pt.pp.K, Nt = pt.pp.Nt, KC = pt.KP / EPC, TP = pt.TP;
                const uint4 *Qhi = reinterpret_cast<const uint4 *>(pt.Qhi);
                const uint4 *Qlo = reinterpret_cast<const uint4 *>(pt.Qlo);
                auto copy_job = [&](const Job &j, bool last) {
                    // the slot is free once the MMAs of job gcopy - NB have completed
                    if (gcopy >= (uint32_t)NB && !wait1(&sm.bempty[bb], bpar ^ 1u, flags)) {
                        failed = true;
                        return;
                    }
                    // the job as the MMA warp needs it (visible to it through bfull: the arrive
                    // below releases this store)
                    sm.jinfo[bb] = (uint32_t)j.k | ((uint32_t)j.nwr << 4) | (last ? 1u << 16 : 0u);
                    // one contiguous block per hi/lo: [nwr/8 groups][KC][8 columns] x 16 bytes
                    const uint32_t bytes = (uint32_t)j.nwr * KC * 16u;
                    mbar_arrive_expect_tx(&sm.bfull[bb], 2u * bytes);
                    const int64_t src = (((int64_t)j.k * (TP / 8) + j.wbeg8 / 8) * KC) * 8;
                    uint4 *slot = B + (size_t)bb * 2 * LKC * bw;
                    bulk_g2s(slot, Qhi + src, bytes, &sm.bfull[bb]);
                    bulk_g2s(slot + (size_t)KC * bw, Qlo + src, bytes, &sm.bfull[bb]);
                    if (++bb == (uint32_t)NB) {
                        bb = 0;
                        bpar ^= 1u;
                    }
                };
                // the quadratic-term jobs come first and need no column ranges: their operands are
                // copied before the tile's A operand and ranges are ready
                // quadratic-term job of detector q: the first QN of the ILE_QCOLS last columns
                for (int q = 0; q < K && !failed; q++, gcopy++) {
                    Job jq{};
                    jq.k = q;
                    jq.wbeg8 = TP - ILE_QCOLS;
                    jq.nwr = QN;
                    copy_job(jq, false);
                }
                if (failed) break;
                if (!wait1(&sm.aready, tiles_done & 1u, flags)) {
                    failed = true;
                    break;
                }
                Det4 lo, hi;
                tile_range(sm.wlo, sm.whi, K, lo, hi);
                JobIter cit(Nt, K, nwcol, lo, hi);
                while (!cit.done && !failed) {
                    const Job j = cit.get();
                    cit.next_from(j);
                    copy_job(j, cit.done);
                    gcopy++;
                }
            }
            if (failed) atomicOr(flags, ILE_FLAG_TIMEOUT);
        }
        __syncwarp();
    } else if (warp == PREF_WARP) {
        // ------------------------------------------------------------------ prefetch warp
        uint32_t tiles_done = 0;
        for (int64_t it = blockIdx.x; it < nitems && !failed; it += gridDim.x, tiles_done++) {
            // the buffer is free once every math thread has read the previous tile's values
            // (they read them before arriving on yready)
            if (tiles_done > 0 && !warp_wait(&sm.yready, (tiles_done - 1) & 1u, flags)) {
                failed = true;
                break;
            }
            int64_t tile;
            const Tc2Point &pt = work_item<BATCH>(one, pts, items, it, tile);
            const PointParams &pp = pt.pp;
            const int64_t N = pt.N;
            // S1 for the tile's samples (rows i * 32 + lane): antenna factors times D_ref / D (1 in the
            // distance-marginalised mode) and fractional window starts, staged as geo[14][TILE]:
            // F_r (4), F_i (4), x0 (4), iota, phi.  Invalid rows repeat the tile's first sample.
#pragma unroll 1
            for (int i = 0; i < TILE / 32; i++) {
                const int r = i * 32 + lane;
                const int64_t p = tile * TILE + r;
                const bool valid = p < N;
                const int64_t src = pt.perm[valid ? p : tile * TILE];
                double th[ILE_NDIM];
                bool finite = true;
#pragma unroll
                for (int d = 0; d < ILE_NDIM; d++) {
                    th[d] = pt.samples[(int64_t)d * N + src];
                    finite = finite && isfinite(th[d]);
                }
                if (!finite || th[5] <= 0.0) {
                    if (valid) atomicOr(flags, ILE_FLAG_NONFINITE);
                    th[0] = th[1] = th[2] = th[3] = th[4] = th[6] = 0.0;
                    th[5] = 1.0;
                }
                const float scale = DM ? 1.f : pp.d_ref / (float)th[5];
                float Fr[ILE_MAX_DET], Fi[ILE_MAX_DET], x0[ILE_MAX_DET];
                ile_sample_geometry(pp, (float)th[0], (float)th[1], (float)th[2], (float)th[6], Fr, Fi, x0);
                bool in_range = true;
#pragma unroll
                for (int k = 0; k < ILE_MAX_DET; k++) {
                    const float fl = floorf(x0[k]);
                    in_range = in_range && (k >= pp.K || (fl >= 0.f && fl + (float)pp.Nt <= (float)(pp.T_ext - 1)));
                }
                if (!in_range && valid) atomicOr(flags, ILE_FLAG_RANGE);
#pragma unroll
                for (int k = 0; k < ILE_MAX_DET; k++) {
                    const bool on = k < pp.K;
                    geo[k * TILE + r] = on ? scale * Fr[k] : 0.f;
                    geo[(4 + k) * TILE + r] = on ? scale * Fi[k] : 0.f;
                    // a sample outside the series gets a harmless placement; the call reports ILE_E_RANGE
                    geo[(8 + k) * TILE + r] = on && in_range ? x0[k] : 0.f;
                }
                geo[12 * TILE + r] = (float)th[3];
                geo[13 * TILE + r] = (float)th[4];
            }
            mbar_arrive(&sm.sready);
        }
        if (failed) atomicOr(flags, ILE_FLAG_TIMEOUT);
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------------ MMA warp
        if (lane == 0) {
            uint32_t gjob = 0, tiles_done = 0;
            // ring positions and phase parities of job gjob (running, no division per job)
            uint32_t bb = 0, bpar = 0, tb = 0, tpar = 0;
            for (int64_t it = blockIdx.x; it < nitems && !failed; it += gridDim.x, tiles_done++) {
                int64_t tile;
                const Tc2Point &pt = work_item<BATCH>(one, pts, items, it, tile);
                const int KP = pt.KP, KC = KP / EPC;
                if (!wait1(&sm.aready, tiles_done & 1u, flags)) {
                    failed = true;
                    break;
                }
                fence_after();
                // shared-memory descriptors: A [KC][TILE rows] chunks (LBO = TILE*16, SBO = 128),
                // B [nwr/8][KC][8] chunks (LBO = 128, SBO = KC*128); a K step (16 BF16 or 8 TF32
                // values, 32 bytes) advances the start address (descriptor bits 0-13, address >> 4)
                // by 2 chunks; the TF32x3 A operand is addressed in TMEM (8 columns per K step)
                const uint64_t a0 = sdesc(smem_u32(A), TILE * 16, 128);
                const uint64_t b0 = sdesc(smem_u32(B), 128, KC * 128);
                const uint64_t a_det = (uint64_t)(2 * KC * TILE * 16) >> 4, a_lo = (uint64_t)(KC * TILE * 16) >> 4;
                const uint64_t b_slot = (uint64_t)(2 * LKC * bw * 16) >> 4, b_lo = (uint64_t)(KC * bw * 16) >> 4;
                const uint64_t a_ks = (uint64_t)(2 * TILE * 16) >> 4, b_ks = (uint64_t)(2 * 128) >> 4;
                // the tile's jobs, in the order the copy warp published them (it enumerates them)
                for (bool last = false; !last && !failed; gjob++) {
                    if (!wait1(&sm.bfull[bb], bpar, flags) || (gjob >= NTBv && !wait1(&sm.tempty[tb], tpar ^ 1u, flags))) {
                        failed = true;
                        break;
                    }
                    fence_after();
                    const uint32_t info = sm.jinfo[bb];
                    const int jk = (int)(info & 15u), nwr = (int)((info >> 4) & 0xFFFu);
                    last = (info >> 16) != 0u;
                    const uint32_t id = idesc(TF32 ? 2 : 1, TILE, nwr);
                    const uint64_t bh = b0 + (uint64_t)bb * b_slot, bl = bh + b_lo;
                    const uint32_t d = tmem + (uint32_t)acol + tb * (uint32_t)bw;
                    uint32_t acc = 0;
                    if constexpr (ATM) {
                        // A in TMEM: hi then lo, KP values each; a K step (8 TF32 or 16 BF16) is 8 columns
                        const int acols = TF32 ? KP : KP / 2;
                        const uint32_t ah = tmem + (uint32_t)(2 * jk * acols), al = ah + (uint32_t)acols;
                        const int nks = acols / 8;
                        for (int pass = 0; pass < 3; pass++) {
                            const uint32_t ad = pass == 2 ? al : ah;
                            const uint64_t bd = pass == 1 ? bl : bh;
                            for (int ks = 0; ks < nks; ks++) {
                                if constexpr (TF32)
                                    mma_tf32_ts(d, ad + (uint32_t)(8 * ks), bd + (uint64_t)ks * b_ks, id, acc);
                                else
                                    mma_bf16_ts(d, ad + (uint32_t)(8 * ks), bd + (uint64_t)ks * b_ks, id, acc);
                                acc = 1;
                            }
                        }
                    } else {
                        const uint64_t ah = a0 + (uint64_t)jk * a_det, al = ah + a_lo;
                        const int nks = KP / 16;
                        for (int pass = 0; pass < 3; pass++) {
                            const uint64_t ad = pass == 2 ? al : ah;
                            const uint64_t bd = pass == 1 ? bl : bh;
                            for (int ks = 0; ks < nks; ks++) {
                                mma_bf16(d, ad + (uint64_t)ks * a_ks, bd + (uint64_t)ks * b_ks, id, acc);
                                acc = 1;
                            }
                        }
                    }
                    mma_commit(&sm.bempty[bb]);
                    mma_commit(&sm.tfull[tb]);
                    if (++bb == (uint32_t)NB) {
                        bb = 0;
                        bpar ^= 1u;
                    }
                    if (++tb == (uint32_t)NTBv) {
                        tb = 0;
                        tpar ^= 1u;
                    }
                }
            }
            if (failed) atomicOr(flags, ILE_FLAG_TIMEOUT);
            // no MMA may still be writing TMEM when it is released (bounded)
            if (gjob > 0)
                mbar_wait_sleep(&sm.tfull[(gjob - 1) % NTBv], ((gjob - 1) / NTBv) & 1u, flags, 0u, SLEEPS, SLEEP_NS);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------ math warps
        const int q4 = warp & 3, g = warp >> 2;
        const int row = q4 * 32 + lane;            // sample row in the tile = TMEM lane
        const uint32_t lane_addr = (uint32_t)(q4 * 32) << 16;
        float *my_row = rows + tid * RS;
        uint32_t tiles_done = 0;
        uint32_t jtb = 0, jtpar = 0;  // TMEM buffer and phase parity of the next job (running)
        uint32_t dmph = 0;            // phases of this quarter's dmx barrier passed (distance marginalisation)
        auto next_job = [&]() {
            if (++jtb == (uint32_t)NTBv) {
                jtb = 0;
                jtpar ^= 1u;
            }
        };
        for (int64_t it = blockIdx.x; it < nitems && !failed; it += gridDim.x, tiles_done++) {
            int64_t tile;
            const Tc2Point &pt = work_item<BATCH>(one, pts, items, it, tile);
            const PointParams &pp = pt.pp;
            const int K = pp.K, M = pp.M, Nt = pp.Nt, KC = pt.KP / 8;  // A-operand units of 8 values
            const int64_t N = pt.N;
            const int *__restrict__ perm = pt.perm;
            double *__restrict__ out = pt.out;
            const int64_t p = tile * TILE + row;
            const bool valid = p < N;
            // ---- S1/S2: geometry (staged by the prefetch warp), harmonics, coefficients
            if (!warp_wait(&sm.sready, tiles_done & 1u, flags)) {
                failed = true;
                break;
            }
            float Fr[ILE_MAX_DET], Fi[ILE_MAX_DET];  // antenna factors times D_ref / D
            int i0[ILE_MAX_DET];
            float wt[ILE_MAX_DET];
#pragma unroll
            for (int k = 0; k < ILE_MAX_DET; k++) {
                Fr[k] = geo[k * TILE + row];
                Fi[k] = geo[(4 + k) * TILE + row];
                const float x0 = geo[(8 + k) * TILE + row];
                const float fl = floorf(x0);
                i0[k] = (int)fl;
                wt[k] = x0 - fl;
            }
            const float iota = geo[12 * TILE + row], phi = geo[13 * TILE + row];
            // grid mode 2 for the adjoint: this sample's window starts and lerp weights
            if (ADJ && g == 0 && valid) {
#pragma unroll
                for (int k = 0; k < ILE_MAX_DET; k++)
                    if (k < K) {
                        pt.sI0[(int64_t)k * N + p] = i0[k];
                        pt.sW[(int64_t)k * N + p] = wt[k];
                    }
            }
            // harmonics: thread g forms modes a = g, g + 4, ... into the shared y table (which
            // reuses the rows area: every thread has passed the previous tile's tdone)
            float2 *ys = reinterpret_cast<float2 *>(rows);  // [M][TILE]
            {
                float cpow[9], spow[9], er[5], ei[5];
                ile_half_angle_powers(iota, cpow, spow);
                ile_phase_powers(phi, er, ei);
#pragma unroll 1
                for (int a = g; a < M; a += NGRP) {
                    float yr, yi;
                    ile_sylm_fast(pp.mode[a], cpow, spow, er, ei, yr, yi);
                    ys[a * TILE + row] = make_float2(yr, yi);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.yready);
            if (!warp_wait(&sm.yready, tiles_done & 1u, flags)) {
                failed = true;
                break;
            }
            {
                // A operand: the K x KC 16-byte chunks of this sample's row (detector k, operand index
                // r = 2a + {0: Re, 1: Im}) are shared round-robin among its four threads
                int k = 0, kc = g;
                while (kc >= KC) {
                    kc -= KC;
                    k++;
                }
#pragma unroll 1
                for (int t = g; t < K * KC; t += NGRP) {
                    const float fr = k == 0 ? Fr[0] : k == 1 ? Fr[1] : k == 2 ? Fr[2] : Fr[3];
                    const float fi = k == 0 ? Fi[0] : k == 1 ? Fi[1] : k == 2 ? Fi[2] : Fi[3];
                    float cv[8];
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        const int a = 4 * kc + e / 2;
                        const float2 y = a < M ? ys[a * TILE + row] : make_float2(0.f, 0.f);
                        cv[e] = fr * y.x - fi * y.y;
                        cv[e + 1] = fr * y.y + fi * y.x;
                    }
                    // grid mode 2 for the adjoint: the coefficients, rows Re c_a at a, Im c_a at M + a
                    if (ADJ && valid) {
#pragma unroll
                        for (int e = 0; e < 8; e++) {
                            const int a = 4 * kc + e / 2;
                            if (a < M) pt.sC[((int64_t)k * 2 * M + ((e & 1) ? M + a : a)) * N + p] = cv[e];
                        }
                    }
                    if constexpr (TF32) {
                        // TMEM lane `row`: hi values at columns 2 k KP + r, lo values KP further
                        uint32_t h[8], l[8];
#pragma unroll
                        for (int e = 0; e < 8; e++) split<false>(cv[e], h[e], l[e]);
                        const uint32_t ta = tmem + lane_addr + (uint32_t)(2 * k * pt.KP + 8 * kc);
                        tmem_st8(ta, h);
                        tmem_st8(ta + (uint32_t)pt.KP, l);
                    } else if constexpr (ATM) {
                        // TMEM lane `row`: BF16 pairs, hi values at columns k KP + r / 2, lo KP / 2 further
                        uint4 h, l;
                        pack_chunk<true>(cv, h, l);
                        const uint32_t ta = tmem + lane_addr + (uint32_t)(k * pt.KP + 4 * kc);
                        tmem_st4(ta, h);
                        tmem_st4(ta + (uint32_t)(pt.KP / 2), l);
                    } else {
                        uint4 h, l;
                        pack_chunk<true>(cv, h, l);
                        A[((size_t)(k * 2) * KC + kc) * TILE + row] = h;
                        A[((size_t)(k * 2 + 1) * KC + kc) * TILE + row] = l;
                    }
                    kc += NGRP;
                    while (kc >= KC) {
                        kc -= KC;
                        k++;
                    }
                }
            }
            // ---- tile column range per detector (invalid rows repeat row 0's sample)
            if (g == 0) {
#pragma unroll
                for (int k = 0; k < ILE_MAX_DET; k++) {
                    if (k < K) {
                        int l = i0[k], h = i0[k];
                        for (int o = 16; o; o >>= 1) {
                            l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
                            h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
                        }
                        if (lane == 0) {
                            sm.wlo[q4][k] = l;
                            sm.whi[q4][k] = h;
                        }
                    }
                }
            }
            if constexpr (ATM) {
                tmem_wait_st();  // this warp's A-operand stores have reached TMEM
                fence_before();
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.aready);  // A operand and column ranges written: the MMAs may start
            if (!warp_wait(&sm.aready, tiles_done & 1u, flags)) {
                failed = true;
                break;
            }
            Det4 lo, hi;
            tile_range(sm.wlo, sm.whi, K, lo, hi);
            const Det4 i0d{i0[0], i0[1], i0[2], i0[3]};
            const Det4f wtd{wt[0], wt[1], wt[2], wt[3]};
            JobIter jit(Nt, K, nwcol, lo, hi);
            // this warp's spread of window offsets per detector, for the single-window jobs (the
            // previous tile's readers of dkr passed tdone before this tile's aready)
#pragma unroll
            for (int k = 0; k < ILE_MAX_DET; k++) {
                if (k < K) {
                    int l = i0d(k) - lo(k), h = l;
                    for (int o = 16; o; o >>= 1) {
                        l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
                        h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
                    }
                    if (lane == 0) sm.dkr[warp][k] = make_int2(l, h);
                }
            }
            __syncwarp();

            // ---- S4 on the tensor cores: the quadratic-term job of detector k leaves in TMEM, for
            // this sample, z = U_k c_k and w = V_k c_k; column (QN / 4) (b % 4) + 4 (b / 4) +
            // {0, 1, 2, 3} holds Re z_b, Im z_b, Re w_b, Im w_b, so thread g's block covers its own
            // modes b = g, g + 4, ... and it forms their part of c^H z + Re(c^T w)
            float aq = 0.f;
            for (int kq = 0; kq < K; kq++) {
                const uint32_t tb = jtb;
                if (!warp_wait(&sm.tfull[tb], jtpar, flags)) {
                    failed = true;
                    break;
                }
                fence_after();
                uint32_t r[32];
                const uint32_t qa = tmem + (uint32_t)acol + tb * (uint32_t)bw + lane_addr + (uint32_t)(QN / 4 * g);
                // the 24 columns of the block (modes b = g + 4 i, i < 6)
                tmem_ld16(qa, *reinterpret_cast<uint32_t(*)[16]>(r));
                tmem_ld8(qa + 16u, *reinterpret_cast<uint32_t(*)[8]>(r + 16));
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.tempty[tb]);
                const float fr = kq == 0 ? Fr[0] : kq == 1 ? Fr[1] : kq == 2 ? Fr[2] : Fr[3];
                const float fi = kq == 0 ? Fi[0] : kq == 1 ? Fi[1] : kq == 2 ? Fi[2] : Fi[3];
                // Re c_b = fr yr - fi yi, Im c_b = fr yi + fi yr;
                // Re(conj(c_b) z_b) + Re(c_b w_b) = Re c_b (Re z_b + Re w_b) + Im c_b (Im z_b - Im w_b)
                float part = 0.f;
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int b = g + 4 * i;
                    if (b < M) {
                        const float2 y = ys[b * TILE + row];
                        const float rc = fmaf(fr, y.x, -fi * y.y), ic = fmaf(fr, y.y, fi * y.x);
                        const float zr = __uint_as_float(r[4 * i]) + __uint_as_float(r[4 * i + 2]);
                        const float zi = __uint_as_float(r[4 * i + 1]) - __uint_as_float(r[4 * i + 3]);
                        part = fmaf(rc, zr, fmaf(ic, zi, part));
                    }
                }
                aq += part;
                next_job();
            }
            if (failed) break;
            aq_s[tid] = 0.25f * aq;
            // everyone is done with the y table before the rows take the TMEM blocks
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.s4done);
            if (!warp_wait(&sm.s4done, tiles_done & 1u, flags)) {
                failed = true;
                break;
            }
            // grid mode 2 for the adjoint: this sample's quadratic term
            if (ADJ && g == 0 && valid)
                pt.sA[p] = aq_s[q4 * 32 + lane] + aq_s[128 + q4 * 32 + lane] + aq_s[256 + q4 * 32 + lane] +
                           aq_s[384 + q4 * 32 + lane];
            // distance-marginalised mode: per-bin terms ln F(D_j, A) with A this sample's quadratic term
            DmargSample dq{};
            if constexpr (DM)
                dq = ile_dmarg_sample(pp.dm, aq_s[q4 * 32 + lane] + aq_s[128 + q4 * 32 + lane] +
                                                 aq_s[256 + q4 * 32 + lane] + aq_s[384 + q4 * 32 + lane]);
            // and no interpolant of this sample yet (its range is empty; read by the sample's
            // four threads after the first chunk's range exchange, which orders this store)
            if (DMREUSE && g == 0) {
                dmc[q4 * 32 + lane] = INFINITY;
                dmc[TILE + q4 * 32 + lane] = -INFINITY;
            }

            // ---- S3/S5: consume the jobs
            float D[JG];
#pragma unroll
            for (int jj = 0; jj < JG; jj++) D[jj] = 0.f;
            float m_run = -INFINITY, s_run = 0.f;
            const int jbeg = g * JG;  // my first bin of a chunk (warp-uniform)
            // distance-marginalised mode: the lane quarter's free word s (0 .. 383) during a chunk's
            // node exchange: word 32 + (s & 1) of the staging row of its thread s / 2 (s < 256),
            // else the aq_s entry of its thread s - 256 (thread t of the quarter: warp 4 (t / 32) + q4)
            auto dm_slot = [&](int s) -> float & {
                if (s < 256) {
                    const int t = s >> 1;
                    return rows[((4 * (t >> 5) + q4) * 32 + (t & 31)) * RS + 32 + (s & 1)];
                }
                const int t = s - 256;
                return aq_s[(4 * (t >> 5) + q4) * 32 + (t & 31)];
            };
            // chunk [j0, j0 + Jc) complete: S5 log-sum-exp update (or the full grid)
            // (sets failed if a distance-marginalised exchange times out)
            auto finish_chunk = [&](int j0, int Jc) {
                if constexpr (DM) {
                    // ln F(D_j, A) of the chunk's bins: one Chebyshev interpolant per sample through 10
                    // table values on a range at least ILE_DM_WMAX wide, kept for the following chunks
                    // of the tile while their data terms stay inside it (a refit otherwise), or
                    // per-bin table reads where a chunk's data terms span more than ILE_DM_WMAX.  The
                    // sample's four threads sit in the four warps of this TMEM lane quarter: each
                    // publishes its bins' range (dmr, one buffer per chunk parity), then, when a
                    // sample of the quarter refits, two or three node values (the two spare words of
                    // its staging row and aq_s, free once the quarter's warps have formed dq), with a
                    // barrier of the quarter after each.  Every decision below is the same in the four
                    // warps (lane l holds the same sample in each), so they pass the same barriers.
                    float lo = INFINITY, hi = -INFINITY;
#pragma unroll
                    for (int jj = 0; jj < JG; jj++)
                        if (jbeg + jj < Jc) {
                            lo = fminf(lo, D[jj]);
                            hi = fmaxf(hi, D[jj]);
                        }
                    float2 *dr = DMREUSE ? dmr + ((j0 / JW) & 1) * NMATH : ls_s;
                    dr[tid] = make_float2(lo, hi);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.dmx[q4]);
                    if (!warp_wait(&sm.dmx[q4], dmph & 1u, flags)) {
                        failed = true;
                        return;
                    }
                    dmph++;
#pragma unroll
                    for (int h = 0; h < NGRP; h++) {
                        const float2 v = dr[(4 * h + q4) * 32 + lane];
                        lo = fminf(lo, v.x);
                        hi = fmaxf(hi, v.y);
                    }
                    const int sl = q4 * 32 + lane;  // the sample's slot in the interpolant store
                    const bool reuse = DMREUSE && lo >= dmc[sl] && hi <= dmc[TILE + sl];  // false for NaN
                    DmRange rg{};
                    float c[ILE_DM_NODES];
                    bool refit = false;
                    if (!reuse) {
                        rg = ile_dm_range_wide(lo, hi);
                        refit = rg.fit;
                    }
                    // (without the store the second exchange also keeps dr = ls_s from being
                    // rewritten before the quarter has read it)
                    if (!DMREUSE || __any_sync(0xffffffffu, refit)) {
                        // the node values of the quarter's refitting samples, spread over its 128
                        // threads: item i = 10 r + n (node n of the warp's r-th refitting lane) is
                        // looked up by thread i mod 128 of the quarter (thread g * 32 + lane) and
                        // stored in the quarter's free word `i` (words 32 and 33 of its staging
                        // rows, then its aq_s entries); rmask is the same in the four warps
                        const unsigned rmask = __ballot_sync(0xffffffffu, refit);
                        const int nitem = ILE_DM_NODES * __popc(rmask);
                        for (int ib = 0; ib < nitem; ib += NMATH / 4) {
                            const int i = ib + g * 32 + lane;
                            const int r = i / ILE_DM_NODES, n = i - r * ILE_DM_NODES;
                            // lane of the (r + 1)-th set bit of rmask: the largest position with
                            // fewer than r + 1 set bits below it
                            int src = 0;
#pragma unroll
                            for (int w = 16; w; w >>= 1)
                                if (__popc(rmask & ((1u << (src + w)) - 1u)) < r + 1) src += w;
                            src = i < nitem ? src : 0;
                            const float mid = __shfl_sync(0xffffffffu, rg.mid, src);
                            const float half = __shfl_sync(0xffffffffu, rg.half, src);
                            DmargSample qs;
                            qs.b = __shfl_sync(0xffffffffu, dq.b, src);
                            qs.inv2b = __shfl_sync(0xffffffffu, dq.inv2b, src);
                            qs.g = __shfl_sync(0xffffffffu, dq.g, src);
                            qs.row = __shfl_sync(0xffffffffu, dq.row, src);
                            qs.big = __shfl_sync(0xffffffffu, dq.big ? 1 : 0, src) != 0;
                            if (i < nitem) dm_slot(i) = ile_dmarg_lnF(pp.dm, qs, fmaf(half, ile_dm_xk[n], mid));
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sm.dmx[q4]);
                        if (!warp_wait(&sm.dmx[q4], dmph & 1u, flags)) {
                            failed = true;
                            return;
                        }
                        dmph++;
                        if (refit) {
                            float f[ILE_DM_NODES];
                            const int rself = __popc(rmask & ((1u << lane) - 1u));
#pragma unroll
                            for (int q = 0; q < ILE_DM_NODES; q++) f[q] = dm_slot(ILE_DM_NODES * rself + q);
                            ile_dm_coeffs(f, c);
                            // the sample's new interpolant for the following chunks: thread g stores
                            // coefficients g, g + 4, g + 8 (thread 0 also the range); read after the
                            // next chunk's range exchange
#pragma unroll
                            for (int q = 0; q < 3; q++)
                                if (DMREUSE && g + 4 * q < ILE_DM_NODES) dmc[(4 + g + 4 * q) * TILE + sl] = c[g + 4 * q];
                            if (DMREUSE && g == 0) {
                                dmc[sl] = rg.mid - rg.half;
                                dmc[TILE + sl] = rg.mid + rg.half;
                                dmc[2 * TILE + sl] = rg.mid;
                                dmc[3 * TILE + sl] = rg.inv_half;
                            }
                        }
                    }
                    if (reuse) {
                        rg.fit = true;
                        rg.mid = dmc[2 * TILE + sl];
                        rg.inv_half = dmc[3 * TILE + sl];
#pragma unroll
                        for (int q = 0; q < ILE_DM_NODES; q++) c[q] = dmc[(4 + q) * TILE + sl];
                    }
                    if (rg.fit) {
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
                if (full_grid == 2) {
                    if (valid) {
                        float *o = pt.grid_f + p * Nt + j0 + jbeg;
                        if (jbeg + JG <= Jc && (Nt & 3) == 0) {
                            // 16 whole bins at a 16-byte boundary (the buffer is 256-byte aligned)
#pragma unroll
                            for (int q = 0; q < JG / 4; q++)
                                reinterpret_cast<float4 *>(o)[q] =
                                    make_float4(D[4 * q], D[4 * q + 1], D[4 * q + 2], D[4 * q + 3]);
                        } else {
#pragma unroll
                            for (int jj = 0; jj < JG; jj++)
                                if (jbeg + jj < Jc) o[jj] = D[jj];
                        }
                    }
                } else if (full_grid) {
                    if (valid) {
                        const double A_n = DM ? 0.0
                                              : (double)(aq_s[q4 * 32 + lane] + aq_s[128 + q4 * 32 + lane] +
                                                         aq_s[256 + q4 * 32 + lane] + aq_s[384 + q4 * 32 + lane]);
                        const int64_t o = (int64_t)perm[p] * Nt + j0 + jbeg;
#pragma unroll
                        for (int jj = 0; jj < JG; jj++)
                            if (jbeg + jj < Jc) out[o + jj] = (double)D[jj] - A_n;
                    }
                } else if (jbeg < Jc) {
                    // all JG bins in the chunk (the usual case), or the first Jc - jbeg of them
                    const bool full = jbeg + JG <= Jc;
                    float mc = -INFINITY;
                    if (full) {
#pragma unroll
                        for (int jj = 0; jj < JG; jj++) mc = fmaxf(mc, D[jj]);
                    } else {
#pragma unroll
                        for (int jj = 0; jj < JG; jj++)
                            if (jbeg + jj < Jc) mc = fmaxf(mc, D[jj]);
                    }
                    if (mc > m_run) {
                        s_run *= __expf(m_run - mc);
                        m_run = mc;
                    }
                    // e^(D - m) = 2^(D log2(e) - m log2(e)): one FMA and one ex2 per bin
                    const float ml2 = m_run * ILE_LOG2E_F;
                    if (full) {
#pragma unroll
                        for (int jj = 0; jj < JG; jj++) s_run += ex2_approx(fmaf(D[jj], ILE_LOG2E_F, -ml2));
                    } else {
#pragma unroll
                        for (int jj = 0; jj < JG; jj++)
                            if (jbeg + jj < Jc) s_run += ex2_approx(fmaf(D[jj], ILE_LOG2E_F, -ml2));
                    }
                }
#pragma unroll
                for (int jj = 0; jj < JG; jj++) D[jj] = 0.f;
            };
            // stage my columns s0 .. s0 + 16 of the job in TMEM buffer tb (the warp loads the 16-column
            // blocks cmin .. cmax; mine: this thread's bins are in the job), then add the lerp
            auto consume = [&](uint32_t tb, int s0, int cmin, int cmax, bool mine, float w, int Jc) {
                const int a0 = s0 & ~15;
                if (cmax >= 0) {
                    const uint32_t taddr = tmem + (uint32_t)acol + tb * (uint32_t)bw + lane_addr;
                    // In a ragged last chunk a thread's second block can start past the job's
                    // window (it holds only bins past the chunk's end, never read); loads stay
                    // inside the buffer, and so inside the TMEM allocation.
                    const int clast = cmax < bw - 16 ? cmax : bw - 16;
                    for (int cb = cmin; cb <= clast; cb += 16) {
                        uint32_t r[16];
                        tmem_ld16(taddr + (uint32_t)cb, r);
                        if (mine && (cb == a0 || cb == a0 + 16)) {
                            if constexpr (RS % 4 == 0) {
                                float4 *dst = reinterpret_cast<float4 *>(my_row + (cb - a0));
#pragma unroll
                                for (int qq = 0; qq < 4; qq++)
                                    dst[qq] = make_float4(__uint_as_float(r[4 * qq]), __uint_as_float(r[4 * qq + 1]),
                                                          __uint_as_float(r[4 * qq + 2]), __uint_as_float(r[4 * qq + 3]));
                            } else {
                                float2 *dst = reinterpret_cast<float2 *>(my_row + (cb - a0));
#pragma unroll
                                for (int qq = 0; qq < 8; qq++)
                                    dst[qq] = make_float2(__uint_as_float(r[2 * qq]), __uint_as_float(r[2 * qq + 1]));
                            }
                        }
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.tempty[tb]);
                if (mine) {
                    const float omw = 1.f - w;
                    const float *src = my_row + (s0 & 15);
                    float vprev = src[0];
                    if (jbeg + JG <= Jc) {
#pragma unroll
                        for (int jj = 0; jj < JG; jj++) {
                            const float v = src[jj + 1];
                            D[jj] = fmaf(omw, vprev, fmaf(w, v, D[jj]));
                            vprev = v;
                        }
                    } else {
#pragma unroll
                        for (int jj = 0; jj < JG; jj++) {
                            if (jbeg + jj < Jc) {
                                const float v = src[jj + 1];
                                D[jj] = fmaf(omw, vprev, fmaf(w, v, D[jj]));
                                vprev = v;
                            }
                        }
                    }
                }
            };
            // every detector's chunk columns fit one window (the usual case for delay-sorted tiles):
            // the jobs are (chunk c, detector k), and a thread's offsets and its warp's block range
            // per detector are the same for every chunk
            bool single = true;
#pragma unroll
            for (int k = 0; k < ILE_MAX_DET; k++)
                if (k < K) single = single && hi(k) - lo(k) + JW + 1 <= nwcol;
            if (single) {
                for (int j0 = 0; j0 < Nt && !failed; j0 += JW) {
                    const int Jc = min(JW, Nt - j0);
                    const bool mine = jbeg < Jc;
#pragma unroll
                    for (int k = 0; k < ILE_MAX_DET; k++) {
                        if (k >= K) break;
                        const uint32_t tb = jtb;
                        if (!warp_wait(&sm.tfull[tb], jtpar, flags)) {
                            failed = true;
                            break;
                        }
                        fence_after();
                        const int shift = jbeg + (lo(k) & 7);  // window start lo_k + j0 rounded down to 8
                        const int2 r = sm.dkr[warp][k];
                        consume(tb, i0d(k) - lo(k) + shift, mine ? (r.x + shift) & ~15 : 0x7fffffff,
                                mine ? ((r.y + shift) & ~15) + 16 : -1, mine, wtd(k), Jc);
                        next_job();
                    }
                    if (failed) break;
                    finish_chunk(j0, Jc);
                }
            } else {
                while (!jit.done) {
                    const Job j = jit.get();
                    const uint32_t tb = jtb;
                    if (!warp_wait(&sm.tfull[tb], jtpar, flags)) {
                        failed = true;
                        break;
                    }
                    fence_after();
                    const int dk = i0d(j.k) - lo(j.k);  // first column of bin 0, relative to the chunk's range
                    const int shift = jbeg + (j.wbeg - j.wbeg8) - j.w * j.step;
                    const int s0 = dk + shift;           // my first column in the window
                    const int a0 = s0 & ~15;
                    bool mine;
                    int cmin, cmax;  // the warp's range of blocks
                    if (j.W == 1) {
                        // one window: every sample reads it; the block range follows from the warp's
                        // offset range ((x & ~15) is monotone)
                        mine = jbeg < j.Jc;
                        const int2 r = sm.dkr[warp][j.k];
                        cmin = mine ? (r.x + shift) & ~15 : 0x7fffffff;
                        cmax = mine ? ((r.y + shift) & ~15) + 16 : -1;
                    } else {
                        const int wsel = min(dk / j.step, j.W - 1);
                        mine = wsel == j.w && jbeg < j.Jc;
                        cmin = mine ? a0 : 0x7fffffff;
                        cmax = mine ? a0 + 16 : -1;
                        for (int o = 16; o; o >>= 1) {
                            cmin = min(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
                            cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
                        }
                    }
                    consume(tb, s0, cmin, cmax, mine, wtd(j.k), j.Jc);
                    next_job();
                    jit.next_from(j);
                    if (j.k == K - 1 && j.w == j.W - 1) {
                        finish_chunk(j.j0, j.Jc);
                        if (failed) break;
                    }
                }
            }
            if (failed) break;
            // ---- merge the four threads' partial log-sum-exps
            ls_s[tid] = make_float2(m_run, s_run);
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.tdone);
            if (!warp_wait(&sm.tdone, tiles_done & 1u, flags)) {
                failed = true;
                break;
            }
            if (g == 0 && valid && !full_grid) {
                // the four threads of this sample: math thread (4h + q4) * 32 + lane, h = 0..3
                float m = -INFINITY, aqs = 0.f;
#pragma unroll
                for (int h = 0; h < NGRP; h++) {
                    const int t = (4 * h + q4) * 32 + lane;
                    m = fmaxf(m, ls_s[t].x);
                    if constexpr (!DM) aqs += aq_s[t];
                }
                float ssum = 0.f;
#pragma unroll
                for (int h = 0; h < NGRP; h++) {
                    const float2 v = ls_s[(4 * h + q4) * 32 + lane];
                    if (v.y > 0.f) ssum += v.y * __expf(v.x - m);
                }
                const double A_n = DM ? 0.0 : (double)aqs;
                const int dst = perm[p];
                out[dst] = (double)m + (double)logf(ssum) - A_n - (double)pp.log_nt;
                // a sample too loud for single precision goes to the FP64 refinement (ile_refine.cu)
                if (!DM && pt.loud.list && fabsf(m) + aqs > pt.loud.thr) ile_loud_append(pt.loud, dst);
            }
        }
        if (failed) atomicOr(flags, ILE_FLAG_TIMEOUT);
    }

    fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

template <int OP>
size_t tc2_smem(int K, int M, int KP, int NB, bool dm = false) {
    const int KC = KP / (OP == OP_TF32_TMEM ? 4 : 8), bw = bw_of(OP);
    (void)M;  // the harmonics table (8 M TILE bytes <= 21.5 KB) fits in the rows area
    const bool a_smem = OP == OP_BF16_SMEM || OP == OP_BF16_SMEM_N;
    return (a_smem ? (size_t)16 * K * 2 * KC * TILE : (size_t)0) + (size_t)16 * NB * 2 * KC * bw +
           sizeof(float) * rstride_of(OP) * NMATH + sizeof(float) * NMATH + sizeof(float2) * NMATH +
           sizeof(float) * 14 * TILE +
           (dm && OP != OP_BF16_SMEM ? sizeof(float) * DMC_ROWS * TILE + sizeof(float2) * 2 * NMATH : (size_t)0);
}
static_assert(8 * ILE_MAX_MODES * TILE <= 4 * RSTRIDE * NMATH, "y table must fit in the rows area");
static_assert(RSTRIDE >= 34, "words 32 and 33 of a staging row carry distance-marginalisation node values");

constexpr size_t SMEM_LIMIT = 227 * 1024 - sizeof(Sm) - 64;

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace
