// ile_adjoint.cu -- hand-written adjoint of the time-marginalised likelihood lnL_t (stages S1-S5):
// the gradient of sum_n g_n lnL_t(n) with respect to every sample's extrinsic parameters
// (ra, dec, psi, iota, phi, D, t_c) and with respect to the inner-product arrays Q, U and V of
// Eq. (eq:QUV).  The paper states no derivative; this is the exact derivative of the function the
// forward kernels compute (FP32 arithmetic, FP64 sums over samples).
//
// With D(n, j) = sum_k [(1 - w_k) G_k(n, i_k + j) + w_k G_k(n, i_k + j + 1)],
// G_k(n, t) = sum_r C_k(r, n) Qp_k(r, t) and lnL_t = LSE_j D(n, j) - A(n) - ln N_t, the window
// softmax pi_j = exp(D_j - LSE) carries the whole backward pass:
//   E_k(r)   = sum_t P_k(t) Qp_k(r, t),  P_k(t) = (1 - w_k) pi_{t - i_k} + w_k pi_{t - i_k - 1}
//              (the pi-weighted interpolated Q: dlnL_t/dC_k(r) = E_k(r) - dA/dC_k(r));
//   S_k      = sum_r C_k(r) sum_t (pi_{t - i_k - 1} - pi_{t - i_k}) Qp_k(r, t)
//              (dlnL_t/dx_k, x_k the fractional window start: the slope of the interpolation);
//   dQp_k(r, t) = sum_n g_n C_k(r, n) P_k(n, t)                       (sample-reduction GEMM);
//   dU_k(a, b) = -1/4 sum_n g_n conj(c_a) c_b,  dV_k(a, b) = -1/4 sum_n g_n c_a c_b.
// The chain rule to theta goes through c_k = (D_ref/D) F_k Y (antenna factors of the wave
// frame, spin-weighted harmonics with d/diota of the Wigner-d polynomial) and x_k through the
// delays dt_k(ra, dec).  The coefficient stage is recomputed, never stored across calls.
//
// Kernels (one call):
//   adj_main   one CTA per tile of NS samples (in delay-sorted order): takes D(n, j) from the
//              fused BF16x3 forward kernel (BF16x3 contexts) or recomputes it with an FP32
//              register-blocked GEMM per 64-column chunk (as the plain forward), takes the
//              window softmax, then per detector a second chunked GEMM
//              [2 NS x 64] x [64 x 2M] gives E and the slope sums; a thread per sample finishes
//              the chain rule and writes g_theta.  pi * g_n goes to HBM for dQ.
//   adj_gq     grid (128-column block, detector, sample split): dQ partials from C and pi*g.
//   adj_guv    grid of sample splits; a thread per (a <= b) mode pair: dU, dV partials.
//   *_reduce   FP64 sums of the partials into the caller's layouts.
#include "ile_internal.cuh"
#include "ile_tcgen05.cuh"

using namespace ile_tc;

namespace {

constexpr int TCOL = 64;                 // columns per chunk in adj_main
constexpr int RMAX = 2 * ILE_MAX_MODES;  // real rows of the contraction (Re rows, then Im rows)
constexpr int RP = 48;                   // rows padded to 3 x 16 for the backward GEMM
constexpr int QT_LD = RP + 1;            // transposed Q chunk row stride (odd: conflict-free)

// Tensor-core forms (BF16x3 contexts).  Shared: 64 samples per adj_main CTA, the TMEM
// accumulator width and the bounded waits.
constexpr int TC_NS = 64;                            // samples per CTA of the main kernel
constexpr uint32_t TC_TMEM_COLS = 64;                // >= RP, power of two
constexpr int TC_SLEEPS = 200000;                    // bounded sleeping waits (x 10 us at most)
constexpr uint32_t TC_SLEEP_NS = 10000;
// E / slope contraction in adj_main: per detector and 64-column chunk, A = [P_E; P_D] (128 rows:
// the pi-weighted interpolation weights of 64 samples and their differences, K = 64 columns, four
// K steps) times B = Qp^T (N = RP rows, K-major), accumulated in TMEM over the chunks.  A is
// single-buffered (every thread packs two of its 16-byte K chunks per chunk), B double-buffered.
constexpr int AM_COLS = 64;
constexpr int AM_KC = AM_COLS / 8;
constexpr int AM_A_BYTES = AM_KC * 128 * 16;  // one of A hi / A lo
constexpr int AM_B_BYTES = AM_KC * RP * 16;   // one of B hi / B lo
constexpr int AM_SMEM = 2 * AM_A_BYTES + 4 * AM_B_BYTES;
// dQ contraction in adj_gq_tc: per chunk of 32 samples (two K steps), A = P^T (128 columns) and
// B = C (RP rows), both operand sets double-buffered.
constexpr int TC_KC = 32 / 8;                        // 16-byte K chunks per chunk
constexpr int TC_A_BYTES = TC_KC * 128 * 16;         // one of A hi / A lo
constexpr int TC_B_BYTES = TC_KC * RP * 16;          // one of B hi / B lo
constexpr int TC_BUF = 2 * TC_A_BYTES + 2 * TC_B_BYTES;
// columns of the transposed split operand: T_ext + one chunk of zeros, so that every chunk that
// starts at or before the last column stays inside the array
__host__ __device__ constexpr int adj_qt_cols(int T) { return T + AM_COLS; }

// d^l_{m,2}(iota) and its derivative d/diota, from the Wigner polynomial in c = cos(iota/2),
// s = sin(iota/2): d/diota c^p s^q = (q c^(p+1) s^(q-1) - p c^(p-1) s^(q+1)) / 2.  Every power is
// at a compile-time index (registers, no local memory): the exponents of mode (l, m) are those the
// host builder lists (ile_wigner_q, q the power of s, p = 2l - q), e^{i m phi} comes from powers
// of e^{i phi}.
template <int L, int MM>
__device__ __forceinline__ void sylm_diota_lm(const ModeTab &md, const float (&cpow)[10], const float (&spow)[10],
                                              const float (&er)[5], const float (&ei)[5], float &yr, float &yi,
                                              float &dr, float &di) {
    constexpr WignerQ w = ile_wigner_q(L, MM);
    float amp = 0.f, damp = 0.f;
#pragma unroll
    for (int t = 0; t < w.n; t++) {
        const int q = w.q[t], p = 2 * L - q;
        const float cf = md.t[t].coef;
        amp += cf * cpow[p] * spow[q];
        float d = 0.f;
        if (q > 0) d += (float)q * cpow[p + 1] * spow[q - 1];
        if (p > 0) d -= (float)p * cpow[p - 1] * spow[q + 1];
        damp += 0.5f * cf * d;
    }
    constexpr int AM = MM < 0 ? -MM : MM;
    const float cs = er[AM], sn = MM < 0 ? -ei[AM] : ei[AM];
    yr = md.norm * amp * cs;
    yi = md.norm * amp * sn;
    dr = md.norm * damp * cs;
    di = md.norm * damp * sn;
}

__device__ __forceinline__ void sylm_and_diota(const ModeTab &md, const float (&cpow)[10], const float (&spow)[10],
                                               const float (&er)[5], const float (&ei)[5], float &yr, float &yi,
                                               float &dr, float &di) {
#define ADJ_LM(L, M)                                                     \
    case (L - 2) * 9 + M + 4:                                            \
        sylm_diota_lm<L, M>(md, cpow, spow, er, ei, yr, yi, dr, di);     \
        return;
    switch ((md.l - 2) * 9 + md.m + 4) {
        ADJ_LM(2, -2) ADJ_LM(2, -1) ADJ_LM(2, 0) ADJ_LM(2, 1) ADJ_LM(2, 2)
        ADJ_LM(3, -3) ADJ_LM(3, -2) ADJ_LM(3, -1) ADJ_LM(3, 0) ADJ_LM(3, 1) ADJ_LM(3, 2) ADJ_LM(3, 3)
        ADJ_LM(4, -4) ADJ_LM(4, -3) ADJ_LM(4, -2) ADJ_LM(4, -1) ADJ_LM(4, 0) ADJ_LM(4, 1) ADJ_LM(4, 2)
        ADJ_LM(4, 3) ADJ_LM(4, 4)
        default:
            yr = yi = dr = di = 0.f;  // 2 <= l <= 4 is checked when the point is set
    }
#undef ADJ_LM
}

__device__ __forceinline__ void half_angle_powers10(float iota, float (&cpow)[10], float (&spow)[10]) {
    float s, c;
    sincosf(0.5f * iota, &s, &c);
    cpow[0] = 1.f;
    spow[0] = 1.f;
#pragma unroll
    for (int i = 1; i < 10; i++) {
        cpow[i] = cpow[i - 1] * c;
        spow[i] = spow[i - 1] * s;
    }
}

__device__ __forceinline__ float dot3(const float *a, const float *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

__device__ __forceinline__ void matvec3(const float *D, const float *x, float *y) {
    y[0] = D[0] * x[0] + D[1] * x[1] + D[2] * x[2];
    y[1] = D[3] * x[0] + D[4] * x[1] + D[5] * x[2];
    y[2] = D[6] * x[0] + D[7] * x[1] + D[8] * x[2];
}

template <int NS, bool TC>
struct MainSmem {
    // row stride of the D / pi rows: odd in the tensor-core form, whose operand build reads them
    // at per-sample offsets
    __host__ __device__ static int ldd(int Nt) { return TC ? Nt + 1 : Nt; }
    static size_t floats(int Nt) {
        const size_t p1 = TC ? 0 : (size_t)RMAX * TCOL + (size_t)NS * (TCOL + 1);
        const size_t p3 = TC ? (size_t)AM_SMEM / 4 : (size_t)TCOL * QT_LD + 2 * (size_t)TCOL * (NS + 4);
        const size_t ep = (size_t)NS * (4 * ILE_MAX_MODES + 1) + 4 + (size_t)ILE_MAX_DET * (ILE_MAX_MODES * (ILE_MAX_MODES + 1) / 2) * 4;
        size_t u = p1 > p3 ? p1 : p3;
        u = u > ep ? u : ep;
        return (size_t)NS * ldd(Nt) + (size_t)RMAX * NS + (size_t)NS * (RMAX + 1) + u;
    }
};

template <int NS, bool TC>
__global__ void __launch_bounds__(TC ? 512 : 256, NS == 32 ? 2 : 1)
    adj_main_kernel(const __grid_constant__ PointParams pp, const float *__restrict__ Qp, const float4 *__restrict__ UV,
                    IleScratch s, const int *__restrict__ perm, const double *__restrict__ samples,
                    const double *__restrict__ g_lnL, int64_t N, float *__restrict__ pig,
                    const float *__restrict__ Din, const uint4 *__restrict__ QThi, const uint4 *__restrict__ QTlo,
                    unsigned *flags, double *__restrict__ g_samples, double *__restrict__ lnl_out) {
    static_assert(!TC || NS == TC_NS, "tensor-core form: 64 samples per CTA");
    // threads per CTA: 16 warps in the tensor-core form (one 219 KB CTA per SM; more warps hide
    // the latency of its D loads, softmax and operand builds), 8 in the CUDA-core form
    constexpr int NT = TC ? 512 : 256, NW = NT / 32;
    constexpr int RS = NS / 16;  // samples per thread in both GEMM micro-tiles (CUDA-core form)
    constexpr int SUB = NT / NS;  // threads per sample in the per-sample stages (mode or pair splits)
    constexpr int PLD = NS + 4;
    constexpr int YLD = 4 * ILE_MAX_MODES + 1;
    extern __shared__ __align__(16) float smem[];
    const int Nt = pp.Nt, M = pp.M, R = 2 * M, T = pp.T_ext, K = pp.K;
    const int LDD = MainSmem<NS, TC>::ldd(Nt);
    float *Ds = smem;                     // [NS][LDD]: D(n, j), then pi(n, j)
    float *Cs = Ds + (size_t)NS * LDD;    // [RMAX][NS]
    float *Es = Cs + RMAX * NS;           // [NS][RMAX + 1]
    float *U1 = Es + NS * (RMAX + 1);     // phase-dependent region
    float *Qs = U1;                       // phase 1: [RMAX][TCOL]
    float *Gs = Qs + RMAX * TCOL;         //          [NS][TCOL + 1]
    float *QsT = U1;                      // phase 3: [TCOL][QT_LD]
    float *PsE = QsT + TCOL * QT_LD;      //          [TCOL][PLD]
    float *PsD = PsE + TCOL * PLD;        //          [TCOL][PLD]
    float *Ys = U1;                       // epilogue: [NS][YLD] (yr, yi, dyr, dyi per mode)
    float4 *UVs = reinterpret_cast<float4 *>(U1 + NS * YLD + ((4 - (NS * YLD) % 4) % 4));  // [K][P]

    __shared__ int i0s[NS];
    __shared__ float ws[NS];
    __shared__ int lo_s[ILE_MAX_DET], hi_s[ILE_MAX_DET];
    __shared__ float Ss[ILE_MAX_DET][NS];
    __shared__ float proj[ILE_MAX_DET][6][NS];
    __shared__ int red[2][NW];
    __shared__ uint16_t pab[ILE_MAX_MODES * (ILE_MAX_MODES + 1) / 2];
    __shared__ uint64_t tc_bfull[2], tc_mma[2], tc_aready[2];
    __shared__ uint32_t tc_tmem;
    __shared__ int tc_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n0 = (int64_t)blockIdx.x * NS;
    const int ns = (int)min((int64_t)NS, N - n0);

    uint32_t tmem = 0;
    if constexpr (TC) {
        if (warp == 0) tmem_alloc(&tc_tmem, TC_TMEM_COLS);
        if (tid == 0) {
            for (int b = 0; b < 2; b++) {
                mbar_init(&tc_bfull[b], 1);
                mbar_init(&tc_mma[b], 1);
                mbar_init(&tc_aready[b], NT);
            }
            tc_abort = 0;
            mbar_init_fence();
        }
        fence_before();
        __syncthreads();
        fence_after();
        tmem = tc_tmem;
    }

    if (LDD == Nt) {
        for (int i = tid; i < NS * Nt; i += NT) Ds[i] = (Din && i < ns * Nt) ? Din[n0 * Nt + i] : 0.f;
    } else {
        // odd row stride: a warp moves 4 rows x 8 float4 (whole 128-byte lines, one per row); lane l
        // stores to row 4 i + l / 8 at column 4 (l % 8) + e, i.e. 32 distinct banks per store
        const int NT4 = Nt / 4, rr = lane >> 3, cc = lane & 7;
        const float4 *src4 = reinterpret_cast<const float4 *>(Din + n0 * Nt);
#pragma unroll 8
        for (int it = warp; it < (NS / 4) * (NT4 / 8); it += NW) {
            const int rg = it / (NT4 / 8), c4 = (it - rg * (NT4 / 8)) * 8 + cc, nn = rg * 4 + rr;
            const float4 v = nn < ns ? src4[(size_t)nn * NT4 + c4] : make_float4(0.f, 0.f, 0.f, 0.f);
            float *d = Ds + nn * LDD + 4 * c4;
            d[0] = v.x;
            d[1] = v.y;
            d[2] = v.z;
            d[3] = v.w;
        }
    }

    auto load_detector = [&](int k) {
        if (tid < NS) {
            int nn = tid < ns ? tid : 0;
            i0s[tid] = s.I0[(int64_t)k * N + n0 + nn];
            ws[tid] = s.W[(int64_t)k * N + n0 + nn];
        }
        for (int i = tid; i < R * NS; i += NT) {
            int r = i / NS, nn = i - r * NS;
            Cs[r * NS + nn] = nn < ns ? s.C[((int64_t)k * R + r) * N + n0 + nn] : 0.f;
        }
    };

    // ---------------------------------------------------------------- phase 1: D(n, j)
    for (int k = 0; k < K; k++) {
        __syncthreads();
        load_detector(k);
        __syncthreads();
        int lo = 0x7fffffff, hi = -0x7fffffff;
        for (int i = tid; i < ns; i += NT) {
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
        for (int w = 1; w < NW; w++) {
            lo = min(lo, red[0][w]);
            hi = max(hi, red[1][w]);
        }
        if (tid == 0) {
            lo_s[k] = lo;
            hi_s[k] = hi;
        }
        if (TC || Din) continue;  // D(n, j) came from the tensor-core forward kernel (always, in that form)
        const int cend = hi + Nt;
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
            for (int nn = warp; nn < ns; nn += NW) {
                const int i0 = i0s[nn];
                const float wt = ws[nn];
                const int jlo = max(0, c0 - 1 - i0), jhi = min(Nt - 1, c0 + TCOL - 1 - i0);
                const float *g = Gs + nn * (TCOL + 1);
                float *d = Ds + (size_t)nn * LDD;
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

    // ---------------------------------------------------------------- phase 2: window softmax
    const double log_nt = log((double)Nt);
    for (int nn = warp; nn < ns; nn += NW) {
        float *d = Ds + (size_t)nn * LDD;
        const int64_t src = perm ? (int64_t)perm[n0 + nn] : n0 + nn;
        float m = -INFINITY;
        for (int j = lane; j < Nt; j += 32) m = fmaxf(m, d[j]);
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        float sum = 0.f;
        for (int j = lane; j < Nt; j += 32) {
            const float e = expf(d[j] - m);
            d[j] = e;  // kept for the normalisation pass
            sum += e;
        }
        for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const float inv = 1.f / sum;
        const float gn = (float)g_lnL[src];
        float *pg = pig ? pig + (size_t)(n0 + nn) * Nt : nullptr;
        for (int j = lane; j < Nt; j += 32) {
            const float p = d[j] * inv;
            d[j] = p;
            if (pg) pg[j] = gn * p;
        }
        if (lnl_out && lane == 0) lnl_out[src] = (double)m + (double)logf(sum) - (double)s.A[n0 + nn] - log_nt;
    }

    // projections of detector k's E on the harmonics: e = sum_a conj(E_a) y_a, with y -> dy/diota,
    // i m y; SUB threads per sample, thread sub taking the modes a = sub, sub + SUB, ...
    // the sample's harmonics and their iota derivatives for this thread's modes a = sub + SUB i,
    // formed once: they serve every detector's projection and the chain rule
    constexpr int YPT = (ILE_MAX_MODES + SUB - 1) / SUB;
    float yh[YPT][4];
    {
        const int nn = tid / SUB, sub = tid % SUB, nv = nn < ns ? nn : 0;
        const int64_t src = perm ? (int64_t)perm[n0 + nv] : n0 + nv;
        const float iota = (float)samples[3 * N + src], phi = (float)samples[4 * N + src];
        float cpow[10], spow[10], er5[5], ei5[5];
        half_angle_powers10(iota, cpow, spow);
        ile_phase_powers(phi, er5, ei5);
#pragma unroll
        for (int i = 0; i < YPT; i++) {
            const int a = sub + SUB * i;
            yh[i][0] = yh[i][1] = yh[i][2] = yh[i][3] = 0.f;
            if (a < M) sylm_and_diota(pp.mode[a], cpow, spow, er5, ei5, yh[i][0], yh[i][1], yh[i][2], yh[i][3]);
        }
    }
    auto project = [&](int k) {
        const int nn = tid / SUB, sub = tid % SUB;
        float er = 0.f, ei = 0.f, gr = 0.f, gi = 0.f, fr = 0.f, fi = 0.f;
        if (nn < ns) {
            const float *E = Es + nn * (RMAX + 1);
#pragma unroll
            for (int i = 0; i < YPT; i++) {
                const int a = sub + SUB * i;
                if (a >= M) break;
                const float yr = yh[i][0], yi = yh[i][1], dr = yh[i][2], di = yh[i][3];
                const float Er = E[a], Ei = E[M + a], mm = (float)pp.mode[a].m;
                er += Er * yr + Ei * yi;
                ei += Er * yi - Ei * yr;
                gr += Er * dr + Ei * di;
                gi += Er * di - Ei * dr;
                // i m y = (-m yi, m yr)
                fr += mm * (-Er * yi + Ei * yr);
                fi += mm * (Er * yr + Ei * yi);
            }
        }
#pragma unroll
        for (int o = SUB / 2; o; o >>= 1) {
            er += __shfl_xor_sync(0xffffffffu, er, o);
            ei += __shfl_xor_sync(0xffffffffu, ei, o);
            gr += __shfl_xor_sync(0xffffffffu, gr, o);
            gi += __shfl_xor_sync(0xffffffffu, gi, o);
            fr += __shfl_xor_sync(0xffffffffu, fr, o);
            fi += __shfl_xor_sync(0xffffffffu, fi, o);
        }
        if (nn < ns && sub == 0) {
            proj[k][0][nn] = er;
            proj[k][1][nn] = ei;
            proj[k][2][nn] = gr;
            proj[k][3][nn] = gi;
            proj[k][4][nn] = fr;
            proj[k][5][nn] = fi;
        }
    };

    // ---------------------------------------------------------------- phase 3: E and slope sums
    if constexpr (TC) {
        // tensor-core form.  Per 64-column chunk, thread (nn, q0) builds the rows nn (P_E) and
        // 64 + nn (P_D) of the 16-byte K chunks q0 and q0 + 4 (8 columns each) of A; thread 0
        // issues 4 K steps x 3 products (hi.hi, hi.lo, lo.hi) into the detector's accumulator and
        // then starts the bulk copies of the next chunk's B (hi, lo) into the other B buffer, so
        // that they land while that chunk's A is built.  A is reused once the chunk's MMAs have
        // completed.  Waits are bounded: a wait that runs out sets the timeout flag and tc_abort,
        // after which no more MMAs are issued (every thread still passes every barrier).  After an
        // abort the other threads skip the MMA waits and may rewrite A while the last committed MMA
        // still reads it: from then on A, B and TMEM hold garbage by design, the call's outputs are
        // discarded and only ILE_E_TIMEOUT is returned; the drain wait on the last commit before
        // TMEM is released stays.
        // thread (nn, q0) builds the K chunks q0, q0 + NT / 64, ... of rows nn and 64 + nn
        constexpr int QSTEP = NT / TC_NS, QPT = (AM_COLS / 8) / QSTEP;
        static_assert(QPT * QSTEP == AM_COLS / 8, "K chunks per thread");
        const int nn = tid & (TC_NS - 1), q0 = tid >> 6;
        uint8_t *tcb = reinterpret_cast<uint8_t *>(U1);
        uint4 *Ah = reinterpret_cast<uint4 *>(tcb), *Al = Ah + AM_A_BYTES / 16;
        const uint32_t id = idesc(1, 128, RP);
        const uint64_t a_ks = (uint64_t)(2 * 128 * 16) >> 4, b_ks = (uint64_t)(2 * RP * 16) >> 4;
        const int TQ8 = adj_qt_cols(T) / 8;
        auto aborted = [&]() { return *(volatile int *)&tc_abort != 0; };
        auto wait = [&](uint64_t *bar, uint32_t parity) {
            if (aborted()) return;
            if (!mbar_wait_sleep(bar, parity, flags, ILE_FLAG_TIMEOUT, TC_SLEEPS, TC_SLEEP_NS)) {
                atomicOr(flags, ILE_FLAG_TIMEOUT);
                tc_abort = 1;
            }
        };
        auto b_hi = [&](int b) { return reinterpret_cast<uint4 *>(tcb + 2 * AM_A_BYTES + b * 2 * AM_B_BYTES); };
        auto copy_b = [&](int b, int k, int c0) {
            uint4 *Bh = b_hi(b), *Bl = Bh + AM_B_BYTES / 16;
            mbar_arrive_expect_tx(&tc_bfull[b], 2u * AM_B_BYTES);
            const size_t off = ((size_t)k * TQ8 + (size_t)(c0 / 8)) * RP;
            bulk_g2s(Bh, QThi + off, AM_B_BYTES, &tc_bfull[b]);
            bulk_g2s(Bl, QTlo + off, AM_B_BYTES, &tc_bfull[b]);
        };
        uint32_t gch = 0;          // chunks issued so far, over all detectors
        int64_t last_commit = -1;  // (thread 0) the last chunk whose MMAs were committed
        for (int k = 0; k < K; k++) {
            __syncthreads();
            load_detector(k);
            __syncthreads();
            // chunks of 64 columns from the tile's first window column (rounded down to 8) to its
            // last lerp partner, inside [0, T_ext)
            const int lo8 = max(lo_s[k], 0) & ~7;
            const int cend = min(hi_s[k] + Nt, T - 1);
            const int nch = cend >= lo8 ? (cend - lo8) / AM_COLS + 1 : 0;
            for (int ci = 0; ci < nch; ci++, gch++) {
                const int bb = (int)(gch & 1u);  // B buffer of this chunk
                const int c0 = lo8 + ci * AM_COLS;
                // A (and the other B buffer) are free once the previous chunk's MMAs have completed
                if (gch >= 1) wait(&tc_mma[0], (gch - 1) & 1u);
                if (tid == 0 && ci == 0 && !aborted()) copy_b(bb, k, c0);  // a detector's first chunk
                {
                    const float wt = ws[nn];
                    const float *pr = Ds + (size_t)nn * LDD;
#pragma unroll
                    for (int it = 0; it < QPT; it++) {
                        const int q = q0 + QSTEP * it;
                        const int j0 = c0 + 8 * q - i0s[nn];  // window bin of the chunk's column 8 q
                        float pe[8], pd[8];
                        float prev = (j0 >= 1 && j0 <= Nt) ? pr[j0 - 1] : 0.f;
#pragma unroll
                        for (int e = 0; e < 8; e++) {
                            const int j = j0 + e;
                            const float cur = (j >= 0 && j < Nt) ? pr[j] : 0.f;
                            pe[e] = (1.f - wt) * cur + wt * prev;
                            pd[e] = prev - cur;
                            prev = cur;
                        }
                        uint4 h, l;
                        pack_chunk<true>(pe, h, l);
                        Ah[q * 128 + nn] = h;
                        Al[q * 128 + nn] = l;
                        pack_chunk<true>(pd, h, l);
                        Ah[q * 128 + TC_NS + nn] = h;
                        Al[q * 128 + TC_NS + nn] = l;
                    }
                }
                // A written: arrive instead of a block barrier, so that thread 0 issues the chunk as
                // soon as the last warp is done
                fence_async_smem();
                mbar_arrive(&tc_aready[0]);
                if (tid == 0) {
                    wait(&tc_aready[0], gch & 1u);
                    wait(&tc_bfull[bb], (gch >> 1) & 1u);
                    if (!aborted()) {
                        fence_after();
                        uint4 *Bh = b_hi(bb), *Bl = Bh + AM_B_BYTES / 16;
                        const uint64_t ah = sdesc(smem_u32(Ah), 128 * 16, 128), al = sdesc(smem_u32(Al), 128 * 16, 128);
                        const uint64_t bh = sdesc(smem_u32(Bh), RP * 16, 128), bl = sdesc(smem_u32(Bl), RP * 16, 128);
                        uint32_t acc = ci > 0 ? 1u : 0u;
                        for (int pass = 0; pass < 3; pass++) {
                            const uint64_t ad = pass == 2 ? al : ah;
                            const uint64_t bd = pass == 1 ? bl : bh;
                            for (int ks = 0; ks < AM_COLS / 16; ks++) {
                                mma_bf16(tmem, ad + (uint64_t)ks * a_ks, bd + (uint64_t)ks * b_ks, id, acc);
                                acc = 1u;
                            }
                        }
                        mma_commit(&tc_mma[0]);
                        last_commit = gch;
                    }
                    // the next chunk's B goes to the other buffer (its previous chunk, gch - 1, has
                    // completed: every thread waited for it at the top of this chunk)
                    if (ci + 1 < nch && !aborted()) copy_b(bb ^ 1, k, c0 + AM_COLS);
                }
            }
            // the detector's sums: rows 0-63 E(r), rows 64-127 the slope terms dE(r)
            if (nch > 0) wait(&tc_mma[0], (gch - 1) & 1u);
            __syncthreads();  // tc_abort is final for this detector: the branch below is uniform
            const bool have = nch > 0 && !aborted();
            fence_after();
            if (warp < 4) {
                const int row = warp * 32 + lane;
                const int sm_ = row & (TC_NS - 1);
                float v[RP];
                if (have) {
                    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
                    for (int cb = 0; cb < RP / 16; cb++) {
                        uint32_t r16[16];
                        tmem_ld16(ta + (uint32_t)(cb * 16), r16);
#pragma unroll
                        for (int i = 0; i < 16; i++) v[cb * 16 + i] = __uint_as_float(r16[i]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < RP; i++) v[i] = 0.f;
                }
                if (row < TC_NS) {
#pragma unroll
                    for (int r = 0; r < RP; r++)
                        if (r < R) Es[sm_ * (RMAX + 1) + r] = v[r];
                } else {
                    float sp = 0.f;
#pragma unroll
                    for (int r = 0; r < RP; r++)
                        if (r < R) sp = fmaf(Cs[r * NS + sm_], v[r], sp);
                    Ss[k][sm_] = sp;
                }
            }
            fence_before();
            __syncthreads();
            project(k);
        }
        // no MMA may still be writing TMEM when it is released (bounded)
        if (tid == 0 && aborted() && last_commit >= 0)
            mbar_wait_sleep(&tc_mma[0], (uint32_t)last_commit & 1u, flags, 0u, TC_SLEEPS, TC_SLEEP_NS);
    } else {
        const int ty = tid >> 4, tx = tid & 15;
        for (int k = 0; k < K; k++) {
            __syncthreads();
            load_detector(k);
            for (int i = tid; i < TCOL * (RP - R); i += 256) {
                int c = i / (RP - R), r = R + i - c * (RP - R);
                QsT[c * QT_LD + r] = 0.f;
            }
            float aE[RS][3], aD[RS][3];
#pragma unroll
            for (int i = 0; i < RS; i++)
#pragma unroll
                for (int m = 0; m < 3; m++) aE[i][m] = aD[i][m] = 0.f;
            const int lo = lo_s[k], cend = hi_s[k] + Nt;
            for (int c0 = lo; c0 <= cend; c0 += TCOL) {
                __syncthreads();
                for (int i = tid; i < R * TCOL; i += 256) {
                    int r = i / TCOL, c = i - r * TCOL;
                    int col = c0 + c;
                    QsT[c * QT_LD + r] = (col >= 0 && col < T) ? Qp[((int64_t)k * R + r) * T + col] : 0.f;
                }
                for (int i = tid; i < NS * TCOL; i += 256) {
                    int c = i / NS, nn = i - c * NS;
                    int j0 = c0 + c - i0s[nn];
                    const float *pr = Ds + (size_t)nn * LDD;
                    float a = (j0 >= 0 && j0 < Nt) ? pr[j0] : 0.f;
                    float b = (j0 >= 1 && j0 <= Nt) ? pr[j0 - 1] : 0.f;
                    float wt = ws[nn];
                    PsE[c * PLD + nn] = (1.f - wt) * a + wt * b;
                    PsD[c * PLD + nn] = b - a;
                }
                __syncthreads();
#pragma unroll 4
                for (int c = 0; c < TCOL; c++) {
                    float pe[RS], pd[RS];
                    if constexpr (RS == 4) {
                        float4 e4 = *reinterpret_cast<const float4 *>(&PsE[c * PLD + ty * 4]);
                        float4 d4 = *reinterpret_cast<const float4 *>(&PsD[c * PLD + ty * 4]);
                        pe[0] = e4.x; pe[1] = e4.y; pe[2] = e4.z; pe[3] = e4.w;
                        pd[0] = d4.x; pd[1] = d4.y; pd[2] = d4.z; pd[3] = d4.w;
                    } else {
#pragma unroll
                        for (int i = 0; i < RS; i++) {
                            pe[i] = PsE[c * PLD + ty * RS + i];
                            pd[i] = PsD[c * PLD + ty * RS + i];
                        }
                    }
                    float q[3];
#pragma unroll
                    for (int m = 0; m < 3; m++) q[m] = QsT[c * QT_LD + tx + 16 * m];
#pragma unroll
                    for (int i = 0; i < RS; i++)
#pragma unroll
                        for (int m = 0; m < 3; m++) {
                            aE[i][m] = fmaf(pe[i], q[m], aE[i][m]);
                            aD[i][m] = fmaf(pd[i], q[m], aD[i][m]);
                        }
                }
            }
            // E to shared memory; slope sum S_k = sum_r C(r) dE(r) reduced over the 16 row lanes
#pragma unroll
            for (int i = 0; i < RS; i++) {
                const int nn = ty * RS + i;
                float sp = 0.f;
#pragma unroll
                for (int m = 0; m < 3; m++) {
                    const int r = tx + 16 * m;
                    if (r < R) {
                        Es[nn * (RMAX + 1) + r] = aE[i][m];
                        sp = fmaf(Cs[r * NS + nn], aD[i][m], sp);
                    }
                }
                for (int o = 8; o; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o);
                if (tx == 0) Ss[k][nn] = sp;
            }
            __syncthreads();
            project(k);
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- epilogue: chain rule to theta
    const int P = M * (M + 1) / 2;
    for (int i = tid; i < K * P; i += NT) UVs[i] = UV[i];
    // mode pairs (a <= b) in the order of the UV table
    for (int i = tid; i < P; i += NT) {
        int a = 0, rest = i;
        while (rest >= M - a) rest -= M - a++;
        pab[i] = (uint16_t)(a | ((a + rest) << 8));
    }
    const int nn = tid / SUB, sub = tid % SUB;  // SUB threads per sample from here on
    if (nn < ns) {
        float *y = Ys + nn * YLD;
#pragma unroll
        for (int i = 0; i < YPT; i++) {
            const int a = sub + SUB * i;
            if (a < M) {
                y[4 * a] = yh[i][0];
                y[4 * a + 1] = yh[i][1];
                y[4 * a + 2] = yh[i][2];
                y[4 * a + 3] = yh[i][3];
            }
        }
    }
    __syncthreads();
    {
        // every thread of a sample runs the preamble; the invalid rows of a ragged tile take
        // sample 0's values and write nothing
        const int nv = nn < ns ? nn : 0;
        const int64_t src = perm ? (int64_t)perm[n0 + nv] : n0 + nv;
        const double gn = g_lnL[src];
        const float ra = (float)samples[src], dec = (float)samples[N + src], psi = (float)samples[2 * N + src];
        const float dist = (float)samples[5 * N + src];
        const float sc = pp.d_ref / dist, sc2 = sc * sc;
        float sg, cg, sd, cd, sp, cp;
        sincosf(pp.gmst - ra, &sg, &cg);
        sincosf(dec, &sd, &cd);
        sincosf(psi, &sp, &cp);
        // wave frame X = cp a + sp b, Y = -sp a + cp b; derivatives in ra (= -d/dg) and dec
        const float av[3] = {-sg, -cg, 0.f}, bv[3] = {-cg * sd, sg * sd, cd};
        const float a_ra[3] = {cg, -sg, 0.f}, b_ra[3] = {-sg * sd, -cg * sd, 0.f};
        const float b_de[3] = {-cg * cd, sg * cd, -sd};
        float X[3], Y[3], Xr[3], Yr[3], Xd[3], Yd[3];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            X[q] = cp * av[q] + sp * bv[q];
            Y[q] = -sp * av[q] + cp * bv[q];
            Xr[q] = cp * a_ra[q] + sp * b_ra[q];
            Yr[q] = -sp * a_ra[q] + cp * b_ra[q];
            Xd[q] = sp * b_de[q];
            Yd[q] = cp * b_de[q];
        }
        const float n_ra[3] = {cd * sg, cd * cg, 0.f}, n_de[3] = {-sd * cg, sd * sg, cd};

        // quadratic-term sums per detector over the mode pairs (U, V pre-doubled off the diagonal)
        float u[ILE_MAX_DET], ui[ILE_MAX_DET], uf[ILE_MAX_DET];
        float vr[ILE_MAX_DET], vi[ILE_MAX_DET], vir[ILE_MAX_DET], vii[ILE_MAX_DET], vfr[ILE_MAX_DET],
            vfi[ILE_MAX_DET];
#pragma unroll
        for (int k = 0; k < ILE_MAX_DET; k++) u[k] = ui[k] = uf[k] = vr[k] = vi[k] = vir[k] = vii[k] = vfr[k] = vfi[k] = 0.f;
        const float *y = Ys + nv * YLD;
        // thread sub takes the pairs p = sub, sub + SUB, ...
        for (int p = sub; p < P; p += SUB) {
            const int a = pab[p] & 0xff, b = pab[p] >> 8;
            {
                const float yar = y[4 * a], yai = y[4 * a + 1], dar = y[4 * a + 2], dai = y[4 * a + 3];
                const float ma = (float)pp.mode[a].m;
                const float ybr = y[4 * b], ybi = y[4 * b + 1], dbr = y[4 * b + 2], dbi = y[4 * b + 3];
                const float mb = (float)pp.mode[b].m;
                // q = conj(y_a) y_b, its iota derivative; pp = y_a y_b, its iota derivative
                const float qr = yar * ybr + yai * ybi, qi = yar * ybi - yai * ybr;
                const float qdr = dar * ybr + dai * ybi + yar * dbr + yai * dbi;
                const float qdi = dar * ybi - dai * ybr + yar * dbi - yai * dbr;
                const float pr = yar * ybr - yai * ybi, pi = yar * ybi + yai * ybr;
                const float pdr = dar * ybr - dai * ybi + yar * dbr - yai * dbi;
                const float pdi = dar * ybi + dai * ybr + yar * dbi + yai * dbr;
                const float dm = mb - ma, sm = ma + mb;
#pragma unroll
                for (int k = 0; k < ILE_MAX_DET; k++) {
                    if (k < K) {
                        const float4 w = UVs[k * P + p];
                        u[k] += w.x * qr - w.y * qi;
                        ui[k] += w.x * qdr - w.y * qdi;
                        uf[k] -= dm * (w.x * qi + w.y * qr);  // Re(U i dm q)
                        const float tr = w.z * pr - w.w * pi, tim = w.z * pi + w.w * pr;  // V p
                        vr[k] += tr;
                        vi[k] += tim;
                        vir[k] += w.z * pdr - w.w * pdi;
                        vii[k] += w.z * pdi + w.w * pdr;
                        vfr[k] -= sm * tim;  // i sm (V p)
                        vfi[k] += sm * tr;
                    }
                }
            }
        }
        // sums over the sample's SUB threads
#pragma unroll
        for (int k = 0; k < ILE_MAX_DET; k++) {
            if (k < K) {
#pragma unroll
                for (int o = SUB / 2; o; o >>= 1) {
                    u[k] += __shfl_xor_sync(0xffffffffu, u[k], o);
                    ui[k] += __shfl_xor_sync(0xffffffffu, ui[k], o);
                    uf[k] += __shfl_xor_sync(0xffffffffu, uf[k], o);
                    vr[k] += __shfl_xor_sync(0xffffffffu, vr[k], o);
                    vi[k] += __shfl_xor_sync(0xffffffffu, vi[k], o);
                    vir[k] += __shfl_xor_sync(0xffffffffu, vir[k], o);
                    vii[k] += __shfl_xor_sync(0xffffffffu, vii[k], o);
                    vfr[k] += __shfl_xor_sync(0xffffffffu, vfr[k], o);
                    vfi[k] += __shfl_xor_sync(0xffffffffu, vfi[k], o);
                }
            }
        }

        float g_ra = 0.f, g_dec = 0.f, g_psi = 0.f, g_iota = 0.f, g_phi = 0.f, g_tc = 0.f, data = 0.f, A = 0.f;
#pragma unroll
        for (int k = 0; k < ILE_MAX_DET; k++) {
            if (k >= K) break;
            const float *D = pp.det_tensor[k];
            float DX[3], DY[3], DXr[3], DYr[3], DXd[3], DYd[3];
            matvec3(D, X, DX);
            matvec3(D, Y, DY);
            matvec3(D, Xr, DXr);
            matvec3(D, Yr, DYr);
            matvec3(D, Xd, DXd);
            matvec3(D, Yd, DYd);
            const float Fr = dot3(X, DX) - dot3(Y, DY), Fi = dot3(X, DY) + dot3(Y, DX);
            const float Fr_ra = dot3(Xr, DX) + dot3(X, DXr) - dot3(Yr, DY) - dot3(Y, DYr);
            const float Fi_ra = dot3(Xr, DY) + dot3(X, DYr) + dot3(Yr, DX) + dot3(Y, DXr);
            const float Fr_de = dot3(Xd, DX) + dot3(X, DXd) - dot3(Yd, DY) - dot3(Y, DYd);
            const float Fi_de = dot3(Xd, DY) + dot3(X, DYd) + dot3(Yd, DX) + dot3(Y, DXd);
            const float dt_ra = -dot3(pp.det_pos_c[k], n_ra), dt_de = -dot3(pp.det_pos_c[k], n_de);
            const float er = proj[k][0][nv], ei = proj[k][1][nv];
            const float gr = proj[k][2][nv], gi = proj[k][3][nv];
            const float fr = proj[k][4][nv], fi = proj[k][5][nv];
            const float S = Ss[k][nv] * pp.fs;
            const float F2 = Fr * Fr + Fi * Fi, Gr = Fr * Fr - Fi * Fi, Gi = 2.f * Fr * Fi;  // |F|^2, F^2
            const float Fvr = Fr * vr[k] - Fi * vi[k], Fvi = Fr * vi[k] + Fi * vr[k];      // F v
            const float gFr = sc * er - 0.5f * sc2 * (Fr * u[k] + Fvr);
            const float gFi = -sc * ei - 0.5f * sc2 * (Fi * u[k] - Fvi);
            g_ra += gFr * Fr_ra + gFi * Fi_ra + S * dt_ra;
            g_dec += gFr * Fr_de + gFi * Fi_de + S * dt_de;
            g_psi += 2.f * (gFr * Fi - gFi * Fr);
            g_iota += sc * (Fr * gr - Fi * gi) - 0.25f * sc2 * (F2 * ui[k] + Gr * vir[k] - Gi * vii[k]);
            g_phi += sc * (Fr * fr - Fi * fi) - 0.25f * sc2 * (F2 * uf[k] + Gr * vfr[k] - Gi * vfi[k]);
            g_tc += S;
            data += sc * (Fr * er - Fi * ei);
            A += 0.25f * sc2 * (F2 * u[k] + Gr * vr[k] - Gi * vi[k]);
        }
        const float g_D = (2.f * A - data) / dist;
        if (g_samples && nn < ns && sub == 0) {
            g_samples[src] = gn * (double)g_ra;
            g_samples[N + src] = gn * (double)g_dec;
            g_samples[2 * N + src] = gn * (double)g_psi;
            g_samples[3 * N + src] = gn * (double)g_iota;
            g_samples[4 * N + src] = gn * (double)g_phi;
            g_samples[5 * N + src] = gn * (double)g_D;
            g_samples[6 * N + src] = gn * (double)g_tc;
        }
    }
    if constexpr (TC) {
        fence_before();
        __syncthreads();
        if (warp == 0) {
            fence_after();
            tmem_dealloc(tmem, TC_TMEM_COLS);
        }
    }
}

// ------------------------------------------------------------------ dQ: sample-reduction GEMM
// dQ_k(r, t) = sum_n C_k(r, n) P_k(n, t), P_k(n, t) = (1 - w) pi(n, t - i0) + w pi(n, t - i0 - 1).
// One CTA per (128-column block, detector, sample split); the samples are consumed in chunks of
// 32 whose raw pi row segments and coefficient columns are brought into shared memory with
// cp.async (zero-filled outside the window), double-buffered: chunk c + 1 is in flight while the
// lerp pass and the register-blocked FMA product of chunk c run.
constexpr int QTB = 128;       // time columns per CTA
constexpr int QNC = 32;        // samples per staged chunk
constexpr int QRW = QTB + 4;   // staged row: pi at t0 - i0 - 1 + m, m = 0 .. QTB (stride padded)

struct GqSmem {
    float raw[2][QNC][QRW];
    float Cc[2][RMAX][QNC];
    float Pc[QNC][QTB];
    int i0c[2][QNC];
    float wc[2][QNC];
};

__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
// 16 bytes, or 16 zero bytes when !valid (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__global__ void __launch_bounds__(256, 2)
    adj_gq_kernel(const __grid_constant__ PointParams pp, const float *__restrict__ pig, IleScratch s, int64_t N,
                  int nsplit, float *__restrict__ part) {
    extern __shared__ __align__(16) uint8_t gq_raw[];
    GqSmem &sm = *reinterpret_cast<GqSmem *>(gq_raw);
    const int Nt = pp.Nt, R = 2 * pp.M, T = pp.T_ext;
    const int t0 = blockIdx.x * QTB, k = blockIdx.y, split = blockIdx.z;
    const int64_t nb = N * split / nsplit, ne = N * (split + 1) / nsplit;
    const int nch = (int)((ne - nb + QNC - 1) / QNC);
    const int tid = threadIdx.x, ry = tid >> 4, tx = tid & 15;
    float acc[3][8];
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[m][j] = 0.f;
    // coefficient rows R .. RMAX - 1 stay zero (the copies write rows < R only)
    for (int i = tid; i < 2 * RMAX * QNC; i += 256) (&sm.Cc[0][0][0])[i] = 0.f;

    // window start and lerp weight of chunk c's sample tid (tid < QNC), 0 beyond the range
    auto load_iw = [&](int c, int &i0v, float &wv) {
        const int64_t n = nb + (int64_t)c * QNC + tid;
        const bool ok = c < nch && n < ne;
        i0v = ok ? s.I0[(int64_t)k * N + n] : 0;
        wv = ok ? s.W[(int64_t)k * N + n] : 0.f;
    };
    auto issue = [&](int c, int b) {
        const int64_t c0 = nb + (int64_t)c * QNC;
        const int nc = (int)min((int64_t)QNC, ne - c0);
        for (int i = tid; i < QNC * (QTB + 1); i += 256) {
            const int j = i / (QTB + 1), m = i - j * (QTB + 1);
            const int idx = t0 - sm.i0c[b][j] - 1 + m;  // pi column
            const bool ok = j < nc && idx >= 0 && idx < Nt;
            cp_async4(&sm.raw[b][j][m], pig + (size_t)(c0 + (j < nc ? j : 0)) * Nt + (ok ? idx : 0), ok);
        }
        for (int i = tid; i < R * QNC; i += 256) {
            const int r = i / QNC, j = i - r * QNC;
            const bool ok = j < nc;
            cp_async4(&sm.Cc[b][r][j], s.C + ((int64_t)k * R + r) * N + c0 + (ok ? j : 0), ok);
        }
    };

    int ri0 = 0;
    float rw = 0.f;
    if (tid < QNC) {
        int a;
        float w;
        load_iw(0, a, w);
        sm.i0c[0][tid] = a;
        sm.wc[0][tid] = w;
        load_iw(1, ri0, rw);
    }
    __syncthreads();
    if (nch > 0) issue(0, 0);
    cp_async_commit();
    for (int c = 0; c < nch; c++) {
        const int b = c & 1;
        if (tid < QNC) {
            sm.i0c[b ^ 1][tid] = ri0;  // chunk c + 1
            sm.wc[b ^ 1][tid] = rw;
            load_iw(c + 2, ri0, rw);
        }
        __syncthreads();  // chunk c + 1's window starts are visible; chunk c - 1's buffers are free
        if (c + 1 < nch) issue(c + 1, b ^ 1);
        cp_async_commit();
        cp_async_wait1();  // this thread's copies of chunk c have landed
        __syncthreads();
        int any = 0;
        for (int i = tid; i < QNC * QTB; i += 256) {
            const int j = i / QTB, col = i - j * QTB;
            const float w = sm.wc[b][j];
            const float a = sm.raw[b][j][col + 1], bb = sm.raw[b][j][col];
            sm.Pc[j][col] = (1.f - w) * a + w * bb;
            const int j0 = t0 + col - sm.i0c[b][j];
            any |= (j0 >= 0 && j0 <= Nt);
        }
        if (!__syncthreads_or(any)) continue;
#pragma unroll 4
        for (int j = 0; j < QNC; j++) {
            const float4 p0 = *reinterpret_cast<const float4 *>(&sm.Pc[j][tx * 4]);
            const float4 p1 = *reinterpret_cast<const float4 *>(&sm.Pc[j][64 + tx * 4]);
            const float pv[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
            for (int m = 0; m < 3; m++) {
                const int r = ry + 16 * m;
                const float cv = r < RMAX ? sm.Cc[b][r][j] : 0.f;
#pragma unroll
                for (int q = 0; q < 8; q++) acc[m][q] = fmaf(cv, pv[q], acc[m][q]);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < 3; m++) {
        const int r = ry + 16 * m;
        if (r >= R) continue;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int t = t0 + (q < 4 ? tx * 4 + q : 64 + tx * 4 + q - 4);
            if (t < T) part[(((int64_t)split * pp.K + k) * R + r) * T + t] = acc[m][q];
        }
    }
}

// Tensor-core form (BF16x3 contexts): the same chunks of 32 samples, staged the same way; per
// chunk the operands A = P^T (128 columns t x 32 samples, K-major: 8 samples per 16 bytes) and
// B = C (RP rows r x 32 samples) are split into BF16 hi / lo and thread 0 issues 2 K steps x 3
// products (hi.hi, hi.lo, lo.hi) into a [128 t x RP r] TMEM accumulator that lives for the whole
// sample split; operand buffers alternate between chunks.  Waits are bounded (a wait that runs
// out sets ILE_FLAG_TIMEOUT and stops further MMAs; every thread still passes every barrier).
static_assert(QNC == 32, "the staging maps one lane to one sample of a chunk");
static_assert(TC_KC * 8 == QNC, "one dQ chunk is TC_KC 16-byte K chunks of samples");
struct GqTcSmem {
    uint8_t ops[2][TC_BUF];  // A hi | A lo | B hi | B lo
    float raw[2][QNC][QRW];
    float Cc[2][RMAX][QNC + 4];  // 16-byte rows: 16-byte staging copies and packing loads
    int i0c[2][QNC];
    int oc[2][QNC];  // offset of pi column t0 - i0 - 1 in its staged row (16-byte staging)
    float wc[2][QNC];
    uint64_t mma[2];
    uint32_t tmem;
    int abort;
};
// 16-byte staging: rows start 16-byte aligned and hold the QTB + 1 values at offsets up to 3
static_assert(QRW % 4 == 0 && QRW >= QTB + 4 && TC_BUF % 16 == 0, "16-byte pi staging");
static_assert((QNC + 4) % 4 == 0 && QNC % 32 == 0, "16-byte coefficient staging");

__global__ void __launch_bounds__(256, 2)
    adj_gq_tc_kernel(const __grid_constant__ PointParams pp, const float *__restrict__ pig, IleScratch s, int64_t N,
                     int nsplit, float *__restrict__ part, unsigned *flags) {
    extern __shared__ __align__(16) uint8_t gq_raw[];
    GqTcSmem &sm = *reinterpret_cast<GqTcSmem *>(gq_raw);
    const int Nt = pp.Nt, R = 2 * pp.M, T = pp.T_ext;
    const int t0 = blockIdx.x * QTB, k = blockIdx.y, split = blockIdx.z;
    // sample splits start on 32-sample boundaries, so that with N a multiple of 4 every chunk's
    // coefficient columns start 16-byte aligned
    auto bound = [&](int sp) { return sp >= nsplit ? N : (N * sp / nsplit) & ~(int64_t)31; };
    const int64_t nb = bound(split), ne = bound(split + 1);
    const int nch = (int)((ne - nb + QNC - 1) / QNC);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) tmem_alloc(&sm.tmem, TC_TMEM_COLS);
    if (tid == 0) {
        mbar_init(&sm.mma[0], 1);
        mbar_init(&sm.mma[1], 1);
        sm.abort = 0;
        mbar_init_fence();
    }
    // coefficient rows R .. RMAX - 1 stay zero (the copies write rows < R only)
    for (int i = tid; i < 2 * RMAX * (QNC + 4); i += 256) (&sm.Cc[0][0][0])[i] = 0.f;
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem;
    auto aborted = [&]() { return *(volatile int *)&sm.abort != 0; };
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (aborted()) return;
        if (!mbar_wait_sleep(bar, parity, flags, ILE_FLAG_TIMEOUT, TC_SLEEPS, TC_SLEEP_NS)) {
            atomicOr(flags, ILE_FLAG_TIMEOUT);
            sm.abort = 1;
        }
    };

    auto load_iw = [&](int c, int &i0v, float &wv) {
        const int64_t n = nb + (int64_t)c * QNC + tid;
        const bool ok = c < nch && n < ne;
        i0v = ok ? s.I0[(int64_t)k * N + n] : 0;
        wv = ok ? s.W[(int64_t)k * N + n] : 0.f;
    };
    // warp w stages the pi row segments of samples w, w + 8, ... (lanes along the row) and the
    // coefficient rows w, w + 8, ... (lanes along the samples)
    // (with N_t a multiple of 4, pi rows are 16-byte aligned: a row segment moves in 16-byte pieces
    // from the 4-aligned column at or below t0 - i0 - 1; every piece lies wholly inside the window
    // [0, N_t) or wholly outside it (zero-filled), and the segment starts oc = (t0 - i0 - 1) mod 4
    // floats into its staged row)
    const bool v16 = (Nt & 3) == 0, c16 = (N & 3) == 0;
    auto issue = [&](int c, int b) {
        const int64_t c0 = nb + (int64_t)c * QNC;
        const int nc = (int)min((int64_t)QNC, ne - c0);
        for (int j = warp; j < QNC; j += 8) {
            const int base = t0 - sm.i0c[b][j] - 1;  // pi column of staged element 0
            const float *row = pig + (size_t)(c0 + (j < nc ? j : 0)) * Nt;
            if (v16) {
                const int sb = base & ~3;  // rounded down to a multiple of 4
                for (int q = lane; q < QRW / 4; q += 32) {
                    const int idx = sb + 4 * q;
                    const bool ok = j < nc && idx >= 0 && idx < Nt;
                    cp_async16(&sm.raw[b][j][4 * q], row + (ok ? idx : 0), ok);
                }
            } else {
                for (int m = lane; m < QTB + 1; m += 32) {
                    const int idx = base + m;
                    const bool ok = j < nc && idx >= 0 && idx < Nt;
                    cp_async4(&sm.raw[b][j][m], row + (ok ? idx : 0), ok);
                }
            }
        }
        if (c16) {
            // coefficient rows in 16-byte pieces of 4 samples (N a multiple of 4, c0 of 32; ne is
            // a multiple of 4 too, so every piece is wholly inside the split or outside it)
            for (int i = tid; i < R * (QNC / 4); i += 256) {
                const int r = i / (QNC / 4), q = i % (QNC / 4);
                const bool ok = 4 * q < nc;
                cp_async16(&sm.Cc[b][r][4 * q], s.C + ((int64_t)k * R + r) * N + c0 + (ok ? 4 * q : 0), ok);
            }
        } else {
            const bool okj = lane < nc;
            for (int r = warp; r < R; r += 8)
                cp_async4(&sm.Cc[b][r][lane], s.C + ((int64_t)k * R + r) * N + c0 + (okj ? lane : 0), okj);
        }
    };

    int ri0 = 0;
    float rw = 0.f;
    if (tid < QNC) {
        int a;
        float w;
        load_iw(0, a, w);
        sm.i0c[0][tid] = a;
        sm.oc[0][tid] = v16 ? ((t0 - a - 1) & 3) : 0;
        sm.wc[0][tid] = w;
        load_iw(1, ri0, rw);
    }
    __syncthreads();
    if (nch > 0) issue(0, 0);
    cp_async_commit();
    const uint32_t id = idesc(1, 128, RP);
    const uint64_t a_ks = (uint64_t)(2 * 128 * 16) >> 4, b_ks = (uint64_t)(2 * RP * 16) >> 4;
    uint32_t issued = 0;  // chunks whose MMAs were issued (uniform over the block)
    for (int c = 0; c < nch; c++) {
        const int b = c & 1;
        if (tid < QNC) {
            sm.i0c[b ^ 1][tid] = ri0;  // chunk c + 1
            sm.oc[b ^ 1][tid] = v16 ? ((t0 - ri0 - 1) & 3) : 0;
            sm.wc[b ^ 1][tid] = rw;
            load_iw(c + 2, ri0, rw);
        }
        __syncthreads();  // chunk c + 1's window starts are visible; chunk c - 1's buffers are free
        if (c + 1 < nch) issue(c + 1, b ^ 1);
        cp_async_commit();
        cp_async_wait1();  // this thread's copies of chunk c have landed
        __syncthreads();
        // chunks whose windows miss the column block contribute nothing
        int any = 0;
        if (tid < QNC) {
            const int lo = t0 - sm.i0c[b][tid], hi = lo + QTB - 1;  // window bins of the block's columns
            any = hi >= 0 && lo <= Nt;
        }
        if (!__syncthreads_or(any)) continue;
        const int ob = (int)(issued & 1u);
        // operand buffer ob is free once the MMAs of the chunk issued two before have completed
        if (issued >= 2) wait(&sm.mma[ob], ((issued - 2) >> 1) & 1u);
        uint4 *Ah = reinterpret_cast<uint4 *>(sm.ops[ob]), *Al = Ah + TC_A_BYTES / 16;
        uint4 *Bh = Al + TC_A_BYTES / 16, *Bl = Bh + TC_B_BYTES / 16;
        // A: thread (t, g) packs P(8 g .. 8 g + 7, t), P(j, t) = (1 - w) pi(t - i0) + w pi(t - i0 - 1)
#pragma unroll
        for (int it = 0; it < 2; it++) {
            const int t = tid & (QTB - 1), g = (tid >> 7) + 2 * it;
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const int j = 8 * g + e;
                const float w = sm.wc[b][j];
                const float *rr = sm.raw[b][j] + sm.oc[b][j];
                v[e] = (1.f - w) * rr[t + 1] + w * rr[t];
            }
            uint4 h, l;
            pack_chunk<true>(v, h, l);
            Ah[g * 128 + t] = h;
            Al[g * 128 + t] = l;
        }
        // B: thread (r, g) packs C(r, 8 g .. 8 g + 7); rows RMAX .. RP - 1 are zero
        if (tid < RP * (QNC / 8)) {
            const int r = tid % RP, g = tid / RP;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
            if (r < RMAX) {
                const float4 *cr = reinterpret_cast<const float4 *>(&sm.Cc[b][r][8 * g]);
                x = cr[0];
                y = cr[1];
            }
            const float v[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
            uint4 h, l;
            pack_chunk<true>(v, h, l);
            Bh[g * RP + r] = h;
            Bl[g * RP + r] = l;
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0 && !aborted()) {
            fence_after();
            const uint64_t ah = sdesc(smem_u32(Ah), 128 * 16, 128), al = sdesc(smem_u32(Al), 128 * 16, 128);
            const uint64_t bh = sdesc(smem_u32(Bh), RP * 16, 128), bl = sdesc(smem_u32(Bl), RP * 16, 128);
            uint32_t acc = issued > 0 ? 1u : 0u;
            for (int pass = 0; pass < 3; pass++) {
                const uint64_t ad = pass == 2 ? al : ah;
                const uint64_t bd = pass == 1 ? bl : bh;
                for (int ks = 0; ks < QNC / 16; ks++) {
                    mma_bf16(tmem, ad + (uint64_t)ks * a_ks, bd + (uint64_t)ks * b_ks, id, acc);
                    acc = 1u;
                }
            }
            mma_commit(&sm.mma[ob]);
        }
        issued++;
    }
    // the split's partial dQ(t, r): wait for the last chunk's MMAs, then one TMEM row per column
    if (issued > 0) wait(&sm.mma[(issued - 1) & 1u], ((issued - 1) >> 1) & 1u);
    __syncthreads();  // the abort flag is final: the branch below is uniform
    const bool have = issued > 0 && !aborted();
    fence_after();
    if (warp < 4) {
        const int t = t0 + warp * 32 + lane;
        float v[RP];
        if (have) {
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
            for (int cb = 0; cb < RP / 16; cb++) {
                uint32_t r16[16];
                tmem_ld16(ta + (uint32_t)(cb * 16), r16);
#pragma unroll
                for (int i = 0; i < 16; i++) v[cb * 16 + i] = __uint_as_float(r16[i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < RP; i++) v[i] = 0.f;
        }
        if (t < T) {
#pragma unroll
            for (int r = 0; r < RP; r++)
                if (r < R) part[(((int64_t)split * pp.K + k) * R + r) * T + t] = v[r];
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}

__global__ void adj_gq_reduce_kernel(int K, int M, int T, int nsplit, const float *__restrict__ part,
                                     double *__restrict__ gQ) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)K * M * T;
    if (i >= total) return;
    const int t = (int)(i % T), a = (int)((i / T) % M), k = (int)(i / ((int64_t)T * M));
    const int R = 2 * M;
    double re = 0.0, im = 0.0;
    for (int sp = 0; sp < nsplit; sp++) {
        re += (double)part[(((int64_t)sp * K + k) * R + a) * T + t];
        im += (double)part[(((int64_t)sp * K + k) * R + M + a) * T + t];
    }
    gQ[2 * i] = re;
    gQ[2 * i + 1] = im;
}

// ------------------------------------------------------------------ dU, dV: weighted pair sums
constexpr int UVC = 64;  // samples per staged chunk

__global__ void __launch_bounds__(256)
    adj_guv_kernel(const __grid_constant__ PointParams pp, const double *__restrict__ samples,
                   const double *__restrict__ g_lnL, int64_t N, int nblk, float *__restrict__ part) {
    __shared__ float2 Yc[UVC][ILE_MAX_MODES + 1];
    __shared__ float Wc[UVC][3 * ILE_MAX_DET];
    const int M = pp.M, K = pp.K, P = M * (M + 1) / 2;
    const int tid = threadIdx.x;
    const int64_t nb = N * blockIdx.x / nblk, ne = N * (blockIdx.x + 1) / nblk;
    // this thread's mode pair (a <= b), p in upper-triangle order
    int pa = 0, pb = 0;
    {
        int p = tid, a = 0;
        while (a < M && p >= M - a) {
            p -= M - a;
            a++;
        }
        pa = a;
        pb = a + p;
    }
    float aUr[ILE_MAX_DET], aUi[ILE_MAX_DET], aVr[ILE_MAX_DET], aVi[ILE_MAX_DET];
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) aUr[k] = aUi[k] = aVr[k] = aVi[k] = 0.f;

    for (int64_t c0 = nb; c0 < ne; c0 += UVC) {
        const int nc = (int)min((int64_t)UVC, ne - c0);
        __syncthreads();
        {
            // four threads per sample of the chunk: each forms the harmonics of modes q, q + 4, ...;
            // the first also the sample's detector weights
            const int j = tid >> 2, q = tid & 3;
            const int64_t n = c0 + j;
            const bool ok = j < nc;
            const float iota = ok ? (float)samples[3 * N + n] : 0.f, phi = ok ? (float)samples[4 * N + n] : 0.f;
            float cpow[9], spow[9], er[5], ei[5];
            ile_half_angle_powers(iota, cpow, spow);
            ile_phase_powers(phi, er, ei);
#pragma unroll 1
            for (int a = q; a < M; a += 4) {
                float yr, yi;
                ile_sylm_fast(pp.mode[a], cpow, spow, er, ei, yr, yi);
                Yc[j][a] = make_float2(yr, yi);
            }
            if (q == 0) {
                float Fr[ILE_MAX_DET], Fi[ILE_MAX_DET], x0[ILE_MAX_DET];
                float g = 0.f, sc2 = 0.f, ra = 0.f, dec = 0.f, psi = 0.f;
                if (ok) {
                    ra = (float)samples[n];
                    dec = (float)samples[N + n];
                    psi = (float)samples[2 * N + n];
                    const float sc = pp.d_ref / (float)samples[5 * N + n];
                    sc2 = sc * sc;
                    g = (float)g_lnL[n];
                }
                ile_sample_geometry(pp, ra, dec, psi, 0.f, Fr, Fi, x0);
                const float wgt = g * sc2;
#pragma unroll
                for (int k = 0; k < ILE_MAX_DET; k++) {
                    if (k < K) {
                        Wc[j][3 * k] = wgt * (Fr[k] * Fr[k] + Fi[k] * Fi[k]);
                        Wc[j][3 * k + 1] = wgt * (Fr[k] * Fr[k] - Fi[k] * Fi[k]);
                        Wc[j][3 * k + 2] = wgt * 2.f * Fr[k] * Fi[k];
                    }
                }
            }
        }
        __syncthreads();
        if (tid < P) {
            for (int j = 0; j < nc; j++) {
                const float2 ya = Yc[j][pa], yb = Yc[j][pb];
                const float qr = ya.x * yb.x + ya.y * yb.y, qi = ya.x * yb.y - ya.y * yb.x;  // conj(y_a) y_b
                const float pr = ya.x * yb.x - ya.y * yb.y, pi = ya.x * yb.y + ya.y * yb.x;  // y_a y_b
#pragma unroll
                for (int k = 0; k < ILE_MAX_DET; k++) {
                    if (k < K) {
                        const float w0 = Wc[j][3 * k], wr = Wc[j][3 * k + 1], wi = Wc[j][3 * k + 2];
                        aUr[k] = fmaf(w0, qr, aUr[k]);
                        aUi[k] = fmaf(w0, qi, aUi[k]);
                        aVr[k] += wr * pr - wi * pi;
                        aVi[k] += wr * pi + wi * pr;
                    }
                }
            }
        }
    }
    if (tid < P) {
        for (int k = 0; k < K; k++) {
            float *o = part + (((int64_t)blockIdx.x * K + k) * P + tid) * 4;
            o[0] = aUr[k];
            o[1] = aUi[k];
            o[2] = aVr[k];
            o[3] = aVi[k];
        }
    }
}

// dU_k(a, b) = -1/4 sum g conj(c_a) c_b and dV_k(a, b) = -1/4 sum g c_a c_b, each entry an
// independent (Re, Im) pair: d/dRe = -1/4 Re(sum), d/dIm = +1/4 Im(sum).
__global__ void adj_guv_reduce_kernel(int K, int M, int nblk, const float *__restrict__ part, double *__restrict__ gU,
                                      double *__restrict__ gV) {
    // one warp per entry (k, p): lane-strided FP64 sums over the blocks, then a fixed xor tree
    // (deterministic; every lane ends with the same sums)
    const int P = M * (M + 1) / 2;
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= K * P) return;
    const int k = i / P, p = i - k * P;
    int a = 0, q = p;
    while (q >= M - a) {
        q -= M - a;
        a++;
    }
    const int b = a + q;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int blk = lane; blk < nblk; blk += 32) {
        const float4 v = *reinterpret_cast<const float4 *>(part + (((int64_t)blk * K + k) * P + p) * 4);
        s[0] += (double)v.x;
        s[1] += (double)v.y;
        s[2] += (double)v.z;
        s[3] += (double)v.w;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1)
#pragma unroll
        for (int c = 0; c < 4; c++) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
    if (lane != 0) return;
    const size_t ab = 2 * (((size_t)k * M + a) * M + b), ba = 2 * (((size_t)k * M + b) * M + a);
    if (gU) {
        gU[ab] = -0.25 * s[0];
        gU[ab + 1] = 0.25 * s[1];
        if (a != b) {
            gU[ba] = -0.25 * s[0];
            gU[ba + 1] = -0.25 * s[1];
        }
    }
    if (gV) {
        gV[ab] = -0.25 * s[2];
        gV[ab + 1] = 0.25 * s[3];
        if (a != b) {
            gV[ba] = -0.25 * s[2];
            gV[ba + 1] = 0.25 * s[3];
        }
    }
}

// Transposed split operand of the tensor-core E contraction: QT[k][c / 8][r][c % 8] (BF16 hi and
// lo of Qp[k][r][c]; zero for r >= 2M and c >= T_ext), one thread per (k, column group, row).
__global__ void adj_qt_kernel(const __grid_constant__ PointParams pp, const float *__restrict__ Qp,
                              uint4 *__restrict__ hi, uint4 *__restrict__ lo) {
    const int T = pp.T_ext, R = 2 * pp.M, TQ8 = adj_qt_cols(T) / 8;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)pp.K * TQ8 * RP) return;
    const int r = (int)(i % RP), cg = (int)((i / RP) % TQ8), k = (int)(i / ((int64_t)RP * TQ8));
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const int c = cg * 8 + e;
        v[e] = (r < R && c < T) ? Qp[((int64_t)k * R + r) * T + c] : 0.f;
    }
    pack_chunk<true>(v, hi[i], lo[i]);
}

template <int NS, bool TC>
cudaError_t launch_main(const PointParams &pp, const float *Qp, const float *UV, IleScratch s, const int *perm,
                        const double *samples, const double *g, int64_t N, float *pig, const float *Din,
                        const void *QThi, const void *QTlo, unsigned *flags, double *g_samples, double *lnl,
                        cudaStream_t st) {
    const size_t smem = sizeof(float) * MainSmem<NS, TC>::floats(pp.Nt) + 16;
    cudaError_t e =
        cudaFuncSetAttribute(adj_main_kernel<NS, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (N + NS - 1) / NS;
    if (TC && !Din) return cudaErrorInvalidValue;  // the tensor-core form takes D(n, j) from the forward kernel
    adj_main_kernel<NS, TC><<<(unsigned)blocks, TC ? 512 : 256, smem, st>>>(pp, Qp, (const float4 *)UV, s, perm, samples, g, N,
                                                                 pig, Din, (const uint4 *)QThi, (const uint4 *)QTlo,
                                                                 flags, g_samples, lnl);
    return cudaGetLastError();
}

}  // namespace

int ile_grad_q_splits(const PointParams &pp, int64_t N, int n_sm) {
    // as many sample splits as keep the grid (column blocks x detectors x splits) within one wave
    // of two CTAs per SM: a partial second wave would leave its few CTAs running alone
    const int tb = (pp.T_ext + QTB - 1) / QTB;
    int64_t want = 2 * (int64_t)n_sm / ((int64_t)tb * pp.K);
    const int64_t most = (N + QNC - 1) / QNC;
    if (want > most) want = most;
    if (want < 1) want = 1;
    return (int)want;
}

int ile_grad_uv_blocks(int64_t N, int n_sm) {
    // four resident blocks per SM (64 registers, 14 KB of shared memory each)
    int64_t b = 4 * (int64_t)n_sm;
    const int64_t most = (N + UVC - 1) / UVC;
    if (b > most) b = most;
    return (int)(b < 1 ? 1 : b);
}

bool ile_grad_tc_ok(const PointParams &pp) {
    // the tensor-core form holds 64 samples' D rows in shared memory and at most RP real rows
    // (and reads them as whole 32-column groups)
    return 2 * pp.M <= RP && pp.Nt % 32 == 0 &&
           sizeof(float) * MainSmem<TC_NS, true>::floats(pp.Nt) + 16 + 12 * 1024 <= 227 * 1024;
}

size_t ile_grad_qt_bytes(const PointParams &pp) { return (size_t)pp.K * (adj_qt_cols(pp.T_ext) / 8) * RP * 16; }

cudaError_t ile_launch_grad_qt(const PointParams &pp, const float *Qp, void *hi, void *lo, cudaStream_t st) {
    const int64_t n = (int64_t)pp.K * (adj_qt_cols(pp.T_ext) / 8) * RP;
    adj_qt_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pp, Qp, (uint4 *)hi, (uint4 *)lo);
    return cudaGetLastError();
}

cudaError_t ile_launch_grad_main(const PointParams &pp, const float *Qp, const float *UV, IleScratch s,
                                 const int *perm, const double *samples, const double *g_lnL, int64_t N, float *pig,
                                 const float *Din, const void *QThi, const void *QTlo, unsigned *flags,
                                 double *g_samples, double *lnl_out, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    if (Din && QThi && QTlo && ile_grad_tc_ok(pp))
        return launch_main<TC_NS, true>(pp, Qp, UV, s, perm, samples, g_lnL, N, pig, Din, QThi, QTlo, flags,
                                        g_samples, lnl_out, st);
    if (pp.Nt <= 256)
        return launch_main<64, false>(pp, Qp, UV, s, perm, samples, g_lnL, N, pig, Din, nullptr, nullptr, flags,
                                      g_samples, lnl_out, st);
    return launch_main<32, false>(pp, Qp, UV, s, perm, samples, g_lnL, N, pig, Din, nullptr, nullptr, flags,
                                  g_samples, lnl_out, st);
}

cudaError_t ile_launch_grad_q(const PointParams &pp, const float *pig, IleScratch s, int64_t N, int nsplit,
                              float *part, double *gQ, bool tc, unsigned *flags, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    dim3 grid((pp.T_ext + QTB - 1) / QTB, pp.K, nsplit);
    cudaError_t e;
    if (tc && 2 * pp.M <= RP) {
        e = cudaFuncSetAttribute(adj_gq_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GqTcSmem));
        if (e != cudaSuccess) return e;
        adj_gq_tc_kernel<<<grid, 256, sizeof(GqTcSmem), st>>>(pp, pig, s, N, nsplit, part, flags);
    } else {
        e = cudaFuncSetAttribute(adj_gq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GqSmem));
        if (e != cudaSuccess) return e;
        adj_gq_kernel<<<grid, 256, sizeof(GqSmem), st>>>(pp, pig, s, N, nsplit, part);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)pp.K * pp.M * pp.T_ext;
    adj_gq_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(pp.K, pp.M, pp.T_ext, nsplit, part, gQ);
    return cudaGetLastError();
}

cudaError_t ile_launch_grad_uv(const PointParams &pp, const double *samples, const double *g_lnL, int64_t N, int nblk,
                               float *part, double *gU, double *gV, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    adj_guv_kernel<<<nblk, 256, 0, st>>>(pp, samples, g_lnL, N, nblk, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int P = pp.M * (pp.M + 1) / 2;
    adj_guv_reduce_kernel<<<(pp.K * P * 32 + 255) / 256, 256, 0, st>>>(pp.K, pp.M, nblk, part, gU, gV);
    return cudaGetLastError();
}
