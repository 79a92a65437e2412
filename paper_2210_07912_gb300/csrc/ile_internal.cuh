// ile_internal.cuh -- shared declarations of the libile CUDA sources (sm_103a only).
//
// Data layout of one intrinsic point in HBM (all owned by the context):
//   Qp   fp32 [K][2M][T_ext]       rows 0..M-1 = Re Q_lm(t), rows M..2M-1 = Im Q_lm(t)
//   UV   fp32 [K][P][4]            P = M(M+1)/2 upper-triangle pairs (a <= b), {Re U, Im U, Re V, Im V}
//                                  with the off-diagonal pairs pre-doubled
//   Qtc  operand tiles of the tensor-core path (see ile_tc.cu)
// Per-sample scratch (sized to the largest N seen):
//   C    fp32 [K][2M][N]           c_klm = (D_ref/D) F_k Y_lm; rows Re then Im
//   I0   int32 [K][N], W fp32 [K][N]: window start index and lerp weight of each detector
//   A    fp32 [N]                  quadratic term <h|h>/2
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ile.h"

#define ILE_PI_F 3.14159265358979f
#define ILE_C_SI 299792458.0

// Device status bits (OR-ed by kernels into a word the host reads after the stream syncs).
#define ILE_FLAG_RANGE 1u
#define ILE_FLAG_NONFINITE 2u
#define ILE_FLAG_TIMEOUT 4u

// d^l_{m,2}(iota) = sum_t coef_t cos(iota/2)^p_t sin(iota/2)^q_t  (at most 3 terms for l <= 4)
struct WignerTerm {
    float coef;
    int p, q;
};

struct ModeTab {
    int l, m;
    float norm;  // sqrt((2l+1)/4pi)
    int nterms;
    WignerTerm t[4];
};

// Distance marginalisation (ile_dmarg.cu): ln F(a, b) = ln int p(D) exp(a x - b x^2) dD,
// x = D_ref / D, p prop. to D^2 on [D_min, D_max], for the data term a and quadratic term b at
// D = D_ref.  Two tables, bilinear:
//   b < b_split: ln F itself on nodes a_i = A0 sinh(tau_i) (tau uniform) x b_k = exp(s_k) (s
//     uniform), interpolated linearly in a and in b (the parts of ln F linear in a and b are
//     reproduced exactly);
//   b >= b_split: H = ln F - E*, E* = a x* - b x*^2 at x* = clip(a / 2b, x_min, x_max), on
//     tau = asinh((u - x_min) / eps) + asinh((u - x_max) / eps) (u = a / 2b; fine near both
//     ends of the distance range) x s = ln b, interpolated linearly in tau and s.
struct DmargParams {
    int on;
    float xmin, xmax, b_split;
    // table 1
    int n1a, n1s;
    float A0, inv_A0, tau1_max, inv_dtau1, s1_lo, ds1;
    const float *t1;   // [n1s][n1a]
    const float2 *a1;  // [n1a] node positions a_i and 1 / (a_{i+1} - a_i)
    // table 2
    int n2t, n2s;
    float eps, inv_eps, tau2_lo, inv_dtau2, s2_lo, inv_ds2;
    const float *t2;   // [n2s][n2t]
    // the same tables as node pairs (t[i], t[i + 1]): one 8-byte load per interval end row
    const float2 *t1p;  // [n1s][n1a]
    const float2 *t2p;  // [n2s][n2t]
};

// Everything a kernel needs about the point besides the big arrays; passed by value.
struct PointParams {
    int K, M, T_ext, Nt;
    float x_offset;   // -t_start*fs - N_t/2: window-start index of a sample is tc*fs + dt*fs + x_offset
    float fs;
    float gmst;
    float d_ref;
    float log_nt;     // ln N_t
    int nearest;      // 1: Q at the nearest sample (window start rounded, interpolation weight 0)
    float det_tensor[ILE_MAX_DET][9];
    float det_pos_c[ILE_MAX_DET][3];  // r_k / c in seconds
    ModeTab mode[ILE_MAX_MODES];
    DmargParams dm;
};

// Per-sample part of the distance-marginalised lookup (b = quadratic term at D_ref > 0).
struct DmargSample {
    float b, inv2b, g;  // g: interpolation weight between the two table rows
    int row;            // first table row (offset in floats)
    bool big;           // table 2
};

__device__ __forceinline__ DmargSample ile_dmarg_sample(const DmargParams &dm, float b) {
    DmargSample q;
    b = fmaxf(b, 1e-30f);
    q.b = b;
    q.inv2b = 0.5f / b;
    q.big = b >= dm.b_split;
    const float s = logf(b);
    if (q.big) {
        float fs = (s - dm.s2_lo) * dm.inv_ds2;
        fs = fminf(fmaxf(fs, 0.f), (float)(dm.n2s - 1) - 1e-3f);
        const int k = (int)fs;
        q.g = fs - (float)k;
        q.row = k * dm.n2t;
    } else {
        float fs = (s - dm.s1_lo) / dm.ds1;
        fs = fminf(fmaxf(fs, 0.f), (float)(dm.n1s - 1) - 1e-3f);
        const int k = (int)fs;
        const float b0 = expf(dm.s1_lo + (float)k * dm.ds1), b1 = expf(dm.s1_lo + (float)(k + 1) * dm.ds1);
        q.g = fminf(fmaxf((b - b0) / (b1 - b0), 0.f), 1.f);
        q.row = k * dm.n1a;
    }
    return q;
}

// asinh for table coordinates, from the fast log2 and reciprocal-square-root units (absolute
// error ~1e-6 in tau; it picks a table node and, for table 2, the weight within a node interval
// of ~0.006 in tau, so the interpolated value moves by a few 1e-4 of one node's step).
__device__ __forceinline__ float ile_asinh_f(float z) {
    const float az = fabsf(z);
    const float s = fmaf(az, az, 1.f);
    return copysignf(__logf(az + s * rsqrtf(s)), z);
}

// ln F(a, b) for one window bin.  Written without branches on the table (the lanes of a warp are
// different samples, whose b can fall in either table): both coordinates' arithmetic is selected.
__device__ __forceinline__ float ile_dmarg_lnF(const DmargParams &dm, const DmargSample &q, float a) {
    const bool big = q.big;
    const float u = a * q.inv2b;
    // table 2: tau = asinh((u - x_min) / eps) + asinh((u - x_max) / eps); table 1: asinh(a / A0)
    const float t1 = ile_asinh_f(big ? (u - dm.xmin) * dm.inv_eps : a * dm.inv_A0);
    const float t2 = ile_asinh_f((u - dm.xmax) * dm.inv_eps);
    float ft = big ? (t1 + t2 - dm.tau2_lo) * dm.inv_dtau2 : (t1 + dm.tau1_max) * dm.inv_dtau1;
    ft = fminf(fmaxf(ft, 0.f), big ? (float)(dm.n2t - 1) - 1e-3f : (float)(dm.n1a - 1) - 1e-3f);
    const int i = (int)ft;
    float f = ft - (float)i;
    if (!big) {
        const float2 nd = __ldg(dm.a1 + i);  // table 1 is linear in a between the nodes a_i, a_{i+1}
        f = fminf(fmaxf((a - nd.x) * nd.y, 0.f), 1.f);
    }
    const float2 *p0 = (big ? dm.t2p : dm.t1p) + q.row + i;
    const float2 lo = __ldg(p0), hi = __ldg(p0 + (big ? dm.n2t : dm.n1a));
    const float h0 = fmaf(f, lo.y - lo.x, lo.x), h1 = fmaf(f, hi.y - hi.x, hi.x);
    const float h = fmaf(q.g, h1 - h0, h0);
    const float xs = fminf(fmaxf(u, dm.xmin), dm.xmax);
    return big ? fmaf(a, xs, -q.b * xs * xs) + h : h;  // table 2 holds ln F - E*
}

// Packed FP32 arithmetic on two lanes (add/mul/fma .rn.f32x2: each lane rounds as its scalar
// IEEE round-to-nearest counterpart, so results equal two scalar operations).
__device__ __forceinline__ float2 ile_f2op_fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
        " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 ile_f2op_add(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " add.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 ile_f2op_mul(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// ---- Distance-marginalised window bins without per-bin table reads.  For one sample (b fixed)
// and one chunk of window bins, ln F(., b) over the chunk's data-term range [a_min, a_max] is its
// degree-9 Chebyshev interpolant through the table values at the 10 Chebyshev points of that
// range (Horner evaluation per bin): 10 table reads per sample and chunk instead of one per bin.
// Where a_max - a_min > ILE_DM_WMAX the bins keep their own table reads.  ln F is analytic in a
// (a cumulant-generating function of x = D_ref / D on [x_min, x_max]).  Against FP64 quadrature of
// ln F for b from 1e-4 to 1e4, the interpolant of the exact function is within 1e-4 of it on
// ranges up to 12 wide (within 5.1e-5 where the data terms of real chunks lie: around 0, b and
// 2b); node values carry the tables' bilinear-interpolation error, which Chebyshev points amplify
// by at most ~2.4 and which varies smoothly along a.  (Degree 11 through 12 points was within
// 2.4e-5; it cost a third more table reads and coefficient arithmetic per chunk.)
constexpr int ILE_DM_NODES = 10;
constexpr float ILE_DM_WMAX = 12.f;

struct DmRange {
    float mid, half, inv_half;
    bool fit;
};

// lo, hi: the chunk's smallest and largest data term (over valid bins) of the sample
__device__ __forceinline__ DmRange ile_dm_range(float lo, float hi) {
    DmRange r;
    r.fit = hi - lo <= ILE_DM_WMAX;  // false for NaN
    r.mid = 0.5f * (lo + hi);
    r.half = fmaxf(0.5f * (hi - lo), 0.5f);  // ranges narrower than 1 are widened to 1 around the middle
    r.inv_half = 1.f / r.half;
    return r;
}

// The same for a fit that later chunks of the sample may reuse: the range is widened to at least
// ILE_DM_WMAX around its middle (the fused kernel keeps the interpolant while a chunk's data terms
// stay inside it).  On ranges that wide the interpolant of the exact ln F stays within 1e-4 of it
// (the bound above); on the benchmarked workload's chunks the per-sample time-marginalised result
// moves by at most 6e-7 against a fit on each chunk's own range.
__device__ __forceinline__ DmRange ile_dm_range_wide(float lo, float hi) {
    DmRange r;
    r.fit = hi - lo <= ILE_DM_WMAX;  // false for NaN
    r.mid = 0.5f * (lo + hi);
    r.half = fmaxf(0.5f * (hi - lo), 0.5f * ILE_DM_WMAX);
    r.inv_half = 1.f / r.half;
    return r;
}

// x_k = cos(pi (k + 1/2) / 10), k = 0 .. 9
static __constant__ float ile_dm_xk[ILE_DM_NODES] = {
    9.876883406e-01f,  8.910065242e-01f,  7.071067812e-01f,  4.539904997e-01f,  1.564344650e-01f,
    -1.564344650e-01f, -4.539904997e-01f, -7.071067812e-01f, -8.910065242e-01f, -9.876883406e-01f};

// Chebyshev point k of the range: mid + half x_k
__device__ __forceinline__ float ile_dm_node(const DmRange &r, int k) { return fmaf(r.half, ile_dm_xk[k], r.mid); }

// Monomial coefficients of T_j: T_0 = 1, T_1 = x, T_{j+1} = 2 x T_j - T_{j-1} (small integers,
// exact in FP32); a[i][j] multiplies x^i in T_j.
struct IleChebMono {
    float a[ILE_DM_NODES][ILE_DM_NODES];
};
__host__ __device__ constexpr IleChebMono ile_cheb_mono() {
    IleChebMono m{};
    m.a[0][0] = 1.f;
    m.a[1][1] = 1.f;
    for (int j = 1; j + 1 < ILE_DM_NODES; j++)
        for (int i = 0; i < ILE_DM_NODES; i++) m.a[i][j + 1] = (i > 0 ? 2.f * m.a[i - 1][j] : 0.f) - m.a[i][j - 1];
    return m;
}

// The interpolant as a polynomial in t = (a - mid) / half: Chebyshev coefficients
// c_j = (2 - [j = 0]) / 10 sum_k f_k T_j(x_k) (using x_{9-k} = -x_k: T_j(x_{9-k}) = (-1)^j T_j(x_k)),
// then m_i = sum_j a[i][j] c_j.  Rounding in c_j stays bounded by the size of T_j on [-1, 1] whatever
// the monomial coefficients; in FP32 the result is within ~1e-5 of the FP64 Clenshaw sum on ranges
// up to ILE_DM_WMAX with |a| < 2000 (above that the FP32 resolution of a itself dominates).
__device__ __forceinline__ void ile_dm_coeffs(const float (&f)[ILE_DM_NODES], float (&m)[ILE_DM_NODES]) {
    constexpr int H = ILE_DM_NODES / 2;
    constexpr float T[ILE_DM_NODES][H] = {
        {1.000000000e-01f, 1.000000000e-01f, 1.000000000e-01f, 1.000000000e-01f, 1.000000000e-01f},
        {1.975376681e-01f, 1.782013048e-01f, 1.414213562e-01f, 9.079809995e-02f, 3.128689301e-02f},
        {1.902113033e-01f, 1.175570505e-01f, 0.000000000e+00f, -1.175570505e-01f, -1.902113033e-01f},
        {1.782013048e-01f, 3.128689301e-02f, -1.414213562e-01f, -1.975376681e-01f, -9.079809995e-02f},
        {1.618033989e-01f, -6.180339887e-02f, -2.000000000e-01f, -6.180339887e-02f, 1.618033989e-01f},
        {1.414213562e-01f, -1.414213562e-01f, -1.414213562e-01f, 1.414213562e-01f, 1.414213562e-01f},
        {1.175570505e-01f, -1.902113033e-01f, 0.000000000e+00f, 1.902113033e-01f, -1.175570505e-01f},
        {9.079809995e-02f, -1.975376681e-01f, 1.414213562e-01f, 3.128689301e-02f, -1.782013048e-01f},
        {6.180339887e-02f, -1.618033989e-01f, 2.000000000e-01f, -1.618033989e-01f, 6.180339887e-02f},
        {3.128689301e-02f, -9.079809995e-02f, 1.414213562e-01f, -1.782013048e-01f, 1.975376681e-01f}};
    constexpr IleChebMono CM = ile_cheb_mono();
    float e[H], o[H], c[ILE_DM_NODES];
#pragma unroll
    for (int k = 0; k < H; k++) {
        e[k] = f[k] + f[ILE_DM_NODES - 1 - k];
        o[k] = f[k] - f[ILE_DM_NODES - 1 - k];
    }
#pragma unroll
    for (int j = 0; j < ILE_DM_NODES; j++) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < H; k++) s = fmaf(T[j][k], (j & 1) ? o[k] : e[k], s);
        c[j] = s;
    }
#pragma unroll
    for (int i = 0; i < ILE_DM_NODES; i++) {
        float s = 0.f;
#pragma unroll
        for (int j = i; j < ILE_DM_NODES; j += 2) s = fmaf(CM.a[i][j], c[j], s);
        m[i] = s;
    }
}

// the interpolant at data term a (Horner in t = (a - mid) / half)
__device__ __forceinline__ float ile_dm_eval(const float (&m)[ILE_DM_NODES], const DmRange &r, float a) {
    const float t = (a - r.mid) * r.inv_half;
    float v = m[ILE_DM_NODES - 1];
#pragma unroll
    for (int i = ILE_DM_NODES - 2; i >= 0; i--) v = fmaf(v, t, m[i]);
    return v;
}

// the same for two bins at once (packed FP32: the results equal two ile_dm_eval calls)
__device__ __forceinline__ float2 ile_dm_eval2(const float (&m)[ILE_DM_NODES], const DmRange &r, float2 a) {
    const float2 t = ile_f2op_mul(ile_f2op_add(a, make_float2(-r.mid, -r.mid)), make_float2(r.inv_half, r.inv_half));
    float2 v = make_float2(m[ILE_DM_NODES - 1], m[ILE_DM_NODES - 1]);
#pragma unroll
    for (int i = ILE_DM_NODES - 2; i >= 0; i--) v = ile_f2op_fma(v, t, make_float2(m[i], m[i]));
    return v;
}

// Adaptive-Cartesian sampler configuration (ile_adapt.cu).
#define ILE_ADAPT_LOG 64
struct IleSamplerParams {
    float lo[ILE_NDIM], hi[ILE_NDIM];  // range of each sampling variable
    unsigned adapt_mask;               // bit d: dimension d is drawn from its histogram
    uint32_t key0, key1;               // Philox key (seed)
    uint32_t point;                    // Philox counter word identifying the intrinsic point
    int sky;                           // 1: variables 0, 1 are the rotated frame's (phi', sin lat')
    float rot[9];                      // rotated frame: columns e1, e2, p (Earth-fixed), row-major
    float gmst;
    unsigned gmm_mask;                 // bits of adapt_mask drawn from a Gaussian mixture (ile_gmm.cu)
    int gmm_pair;                      // 1: variables 0 and 1 drawn together from the correlated pair mixture
};

// One dimension's Gaussian mixture in FP64 (the adapted state) and its sampler form in FP32.
struct IleGmm {
    int C;
    double lo, hi;
    double w[ILE_GMM_MAX], mu[ILE_GMM_MAX], sigma[ILE_GMM_MAX];
    double n;  // samples the mixture has been trained on
};
struct IleGmmTab {
    uint64_t cw[ILE_GMM_MAX + 1];  // integer cumulative weights, 2^32 scale
    float mu[ILE_GMM_MAX], sig[ILE_GMM_MAX];
    float p1[ILE_GMM_MAX];    // Phi(z_lo): mass of the normal below the range
    float q2[ILE_GMM_MAX];    // Phi(-z_hi): mass above the range
    float dm[ILE_GMM_MAX];    // Z = Phi(z_hi) - Phi(z_lo): mass inside
    float coef[ILE_GMM_MAX];  // ln(w_c / (sqrt(2 pi) sigma_c Z_c))
    int C;
};

// The sky pair's correlated mixture in FP64 (the adapted state): component c has weight w[c], mean
// mu[c] and covariance cov[c] = {S00, S01, S11}, a bivariate normal truncated to the rectangle
// [lo0, hi0] x [lo1, hi1] of sampling variables 0 and 1.
struct IleGmm2 {
    int C;
    double lo[2], hi[2];
    double w[ILE_GMM_MAX], mu[ILE_GMM_MAX][2], cov[ILE_GMM_MAX][3];
    double n;
};
// Its sampler form in FP32: integer weight table; per component the mean, the Cholesky factor
// L = {l00, l10, l11} of the covariance, per whitened axis j the box [blo, bhi] that holds the
// image of the rectangle as Phi(blo) (p1), Phi(-bhi) (q2) and Phi(bhi) - Phi(blo) (dm), the inverse
// covariance {i00, i01, i11} and ln(w_c / (2 pi sqrt(det) Z_c)) with Z_c the component's mass in
// the rectangle.
struct IleGmm2Tab {
    uint64_t cw[ILE_GMM_MAX + 1];
    float mu[ILE_GMM_MAX][2], L[ILE_GMM_MAX][3], icov[ILE_GMM_MAX][3];
    float p1[ILE_GMM_MAX][2], q2[ILE_GMM_MAX][2], dm[ILE_GMM_MAX][2];
    float coef[ILE_GMM_MAX];
    int C;
};

// Rotated-frame basis from a pole vector (host; see ile.h): returns false for a zero vector.
bool ile_sky_frame(const double pole[3], float rot[9]);

// One point of a batched adaptive run (ile_batch.cu): its sampler and the location of its
// samples in the batch's concatenated per-sample arrays (theta and bins at ILE_NDIM * off,
// laid out [7][N]; everything else at off).
struct IleBatchPoint {
    IleSamplerParams sp;
    double eps;
    int64_t N, off;
    float gmst;
};

// Per-sample geometry: antenna factors and window placement of detector k.
__device__ __forceinline__ void ile_sample_geometry(const PointParams &pp, float ra, float dec, float psi, float tc,
                                                    float Fr[ILE_MAX_DET], float Fi[ILE_MAX_DET],
                                                    float x0[ILE_MAX_DET]) {
    float sg, cg, sd, cd, sp, cp;
    sincosf(pp.gmst - ra, &sg, &cg);
    sincosf(dec, &sd, &cd);
    sincosf(psi, &sp, &cp);
    float X0 = -cp * sg - sp * cg * sd, X1 = -cp * cg + sp * sg * sd, X2 = sp * cd;
    float Y0 = sp * sg - cp * cg * sd, Y1 = sp * cg + cp * sg * sd, Y2 = cp * cd;
    float n0 = cd * cg, n1 = -cd * sg, n2 = sd;
#pragma unroll
    for (int k = 0; k < ILE_MAX_DET; k++) {
        if (k >= pp.K) break;
        const float *D = pp.det_tensor[k];
        float DX0 = D[0] * X0 + D[1] * X1 + D[2] * X2;
        float DX1 = D[3] * X0 + D[4] * X1 + D[5] * X2;
        float DX2 = D[6] * X0 + D[7] * X1 + D[8] * X2;
        float DY0 = D[0] * Y0 + D[1] * Y1 + D[2] * Y2;
        float DY1 = D[3] * Y0 + D[4] * Y1 + D[5] * Y2;
        float DY2 = D[6] * Y0 + D[7] * Y1 + D[8] * Y2;
        Fr[k] = (X0 * DX0 + X1 * DX1 + X2 * DX2) - (Y0 * DY0 + Y1 * DY1 + Y2 * DY2);
        Fi[k] = (X0 * DY0 + X1 * DY1 + X2 * DY2) + (Y0 * DX0 + Y1 * DX1 + Y2 * DX2);
        float dt = -(pp.det_pos_c[k][0] * n0 + pp.det_pos_c[k][1] * n1 + pp.det_pos_c[k][2] * n2);
        x0[k] = (tc + dt) * pp.fs + pp.x_offset;
        // nearest-sample mode: bin j reads sample rint(x0 + j) = rint(x0) + j with weight 0
        if (pp.nearest) x0[k] = rintf(x0[k]);
    }
}

// Spin-weighted harmonic _{-2}Y_lm(iota, phi) of mode a.
__device__ __forceinline__ void ile_sylm(const ModeTab &md, const float cpow[9], const float spow[9], float phi,
                                         float &yr, float &yi) {
    float amp = 0.f;
    for (int t = 0; t < md.nterms; t++) amp += md.t[t].coef * cpow[md.t[t].p] * spow[md.t[t].q];
    amp *= md.norm;
    float s, c;
    sincosf((float)md.m * phi, &s, &c);
    yr = amp * c;
    yi = amp * s;
}

// The same harmonics with every power at a compile-time index (registers, no local memory) and
// e^{i m phi} from powers of e^{i phi}: the exponents of the terms of d^l_{m,2} that the host
// builder (wigner_terms) lists, in its order, for the 21 modes with 2 <= l <= 4.
struct WignerQ {
    int n;
    int q[4];  // power of s = sin(iota/2) of each term; the power of c is 2l - q
};
__host__ __device__ constexpr WignerQ ile_wigner_q(int l, int m) {
    WignerQ w{0, {0, 0, 0, 0}};
    for (int sp = 0; sp <= 2 * l; sp++) {
        const int twok = sp + 2 - m;
        if (twok < 0 || (twok & 1)) continue;
        const int k = twok / 2;
        if (l + 2 - k < 0 || l - m - k < 0 || k + m - 2 < 0) continue;
        if (w.n < 4) w.q[w.n++] = sp;
    }
    return w;
}

template <int L, int M>
__device__ __forceinline__ void ile_sylm_lm(const ModeTab &md, const float (&cpow)[9], const float (&spow)[9],
                                            const float (&er)[5], const float (&ei)[5], float &yr, float &yi) {
    constexpr WignerQ w = ile_wigner_q(L, M);
    float amp = 0.f;
#pragma unroll
    for (int t = 0; t < w.n; t++) amp += md.t[t].coef * cpow[2 * L - w.q[t]] * spow[w.q[t]];
    amp *= md.norm;
    constexpr int AM = M < 0 ? -M : M;
    yr = amp * er[AM];
    yi = M < 0 ? -amp * ei[AM] : amp * ei[AM];
}

// e^{i m phi}, m = 0..4
__device__ __forceinline__ void ile_phase_powers(float phi, float (&er)[5], float (&ei)[5]) {
    er[0] = 1.f;
    ei[0] = 0.f;
    sincosf(phi, &ei[1], &er[1]);
    er[2] = er[1] * er[1] - ei[1] * ei[1];
    ei[2] = 2.f * er[1] * ei[1];
    er[3] = er[2] * er[1] - ei[2] * ei[1];
    ei[3] = er[2] * ei[1] + ei[2] * er[1];
    er[4] = er[2] * er[2] - ei[2] * ei[2];
    ei[4] = 2.f * er[2] * ei[2];
}

__device__ __forceinline__ void ile_sylm_fast(const ModeTab &md, const float (&cpow)[9], const float (&spow)[9],
                                              const float (&er)[5], const float (&ei)[5], float &yr, float &yi) {
#define ILE_LM(L, M)                                            \
    case (L - 2) * 9 + M + 4:                                   \
        ile_sylm_lm<L, M>(md, cpow, spow, er, ei, yr, yi);      \
        return;
    switch ((md.l - 2) * 9 + md.m + 4) {
        ILE_LM(2, -2) ILE_LM(2, -1) ILE_LM(2, 0) ILE_LM(2, 1) ILE_LM(2, 2)
        ILE_LM(3, -3) ILE_LM(3, -2) ILE_LM(3, -1) ILE_LM(3, 0) ILE_LM(3, 1) ILE_LM(3, 2) ILE_LM(3, 3)
        ILE_LM(4, -4) ILE_LM(4, -3) ILE_LM(4, -2) ILE_LM(4, -1) ILE_LM(4, 0) ILE_LM(4, 1) ILE_LM(4, 2)
        ILE_LM(4, 3) ILE_LM(4, 4)
        default:
            yr = yi = 0.f;  // 2 <= l <= 4 is checked when the point is set
    }
#undef ILE_LM
}

__device__ __forceinline__ void ile_half_angle_powers(float iota, float cpow[9], float spow[9]) {
    float s, c;
    sincosf(0.5f * iota, &s, &c);
    cpow[0] = 1.f;
    spow[0] = 1.f;
#pragma unroll
    for (int i = 1; i < 9; i++) {
        cpow[i] = cpow[i - 1] * c;
        spow[i] = spow[i - 1] * s;
    }
}

// FP64 description of a point for the refinement of loud samples (ile_refine.cu).
struct Mode64 {
    int l, m, nterms;
    double norm;     // sqrt((2l+1)/4pi)
    double coef[4];  // d^l_{m,2}(iota) = sum_t coef_t cos(iota/2)^p_t sin(iota/2)^q_t
    int p[4], q[4];
};
struct Refine64 {
    int K, M, Nt, T_ext;
    double fs, t_start, gmst, d_ref, log_nt;
    float thr;    // a window bin's data term is recomputed in FP64 when |D_j| exceeds this
    int nearest;  // 1: Q at the nearest sample
    double det_tensor[ILE_MAX_DET][9];
    double det_pos[ILE_MAX_DET][3];  // metres
    Mode64 mode[ILE_MAX_MODES];
};

// Device list of loud samples: list[0] = count, then (point, caller index) pairs at list[1 + 2 i],
// list[2 + 2 i], i < cap (the list holds 2 cap + 1 ints).  A fast kernel appends a sample when
// |max_j D(n, j)| + A(n) > thr (list == nullptr: no list); point identifies the intrinsic point in a
// batched run (0 otherwise).  The count is reset before every launch that fills the list; appends
// past cap are dropped.
struct LoudList {
    int *list;
    float thr;
    int point;
    int64_t cap;
};
__device__ __forceinline__ void ile_loud_append(const LoudList &l, int n) {
    const int i = atomicAdd(l.list, 1);
    if (i < l.cap) {
        l.list[1 + 2 * i] = l.point;
        l.list[2 + 2 * i] = n;
    }
}
// One point of a batched refinement (ile_refine.cu): its FP64 description and arrays, its samples
// [7][N] and its lnL_t [N].
struct RefinePoint {
    Refine64 r;
    const double2 *Q64, *U64, *V64;
    const float *Qp;
    const double *samples;
    int64_t N;
    double *out;
};

// One intrinsic point as seen by the fused tensor-core kernel (ile_tc2_kernel.cuh).
struct Tc2Point {
    PointParams pp;
    const void *Qhi, *Qlo;  // split operand tiles of Q (ile_tc.cu layout)
    const float *UV;        // [K][P][4]
    const double *samples;  // SoA [7][N]
    const int *perm;        // [N] processing order -> caller index
    double *out;            // [N]
    float *grid_f;          // grid mode 2: data term D(n, j) in processing order [N][N_t]
    // grid mode 2 (may be null): the per-sample coefficients C [K][2M][N], window starts I0 [K][N],
    // lerp weights W [K][N] and quadratic term A [N] in processing order, as ile_prep_kernel writes them
    float *sC;
    int *sI0;
    float *sW, *sA;
    int64_t N;
    int TP, KP;
    LoudList loud;          // loud samples for the FP64 refinement (single-point launches)
};

// ------------------------------------------------------------------ host-side launch wrappers
// (defined in the .cu files; all take the context's stream)
struct IleScratch {
    float *C;
    int *I0;
    float *W;
    float *A;
};

cudaError_t ile_launch_prep(const PointParams &pp, const float *UV, const double *samples, const int *perm, int64_t N,
                            IleScratch s, unsigned *flags, cudaStream_t st);
cudaError_t ile_launch_plain(const PointParams &pp, const float *Qp, IleScratch s, const int *perm, int64_t N,
                             double *out, int full_grid, LoudList loud, unsigned *flags, cudaStream_t st);
// FP64 refinement of the samples in list (ile_refine.cu): lnL_t recomputed into out (caller order)
cudaError_t ile_launch_refine(const Refine64 &P, const double2 *Q64, const double2 *U64, const double2 *V64,
                              const float *Qp, const double *samples, int64_t N, const int *list, int64_t cap,
                              double *out, unsigned *flags, int n_sm, cudaStream_t st);
cudaError_t ile_launch_batch_refine(const RefinePoint *pts, int64_t n_total, const int *list, int64_t cap,
                                    unsigned *flags, int n_sm, cudaStream_t st);
// FP64 description of a point (ile_api.cu) and the refinement threshold of a precision
bool ile_refine_params(int n_det, int n_modes, const int *lm, const double *det_tensor, const double *det_pos_m,
                       int T_ext, double t_start_s, double fs_hz, int n_window, double gmst_rad, double d_ref_mpc,
                       Refine64 &r);
float ile_refine_threshold(int prec);
// delay-bucket sort (ile_sort.cu): keys [N], buckets [ile_sort_key_buckets()], perm [N]
size_t ile_sort_key_buckets();
cudaError_t ile_launch_sort(const PointParams &pp, const double *samples, int64_t N, int *keys, int *buckets,
                            int *perm, cudaStream_t st);
// the same order with equal keys kept in the caller's order (deterministic; the adjoint's
// sample sums run in this order): work holds ile_sort_stable_work_ints(N) ints
size_t ile_sort_stable_work_ints(int64_t N);
cudaError_t ile_launch_sort_stable(const PointParams &pp, const double *samples, int64_t N, int *keys, int *work,
                                   int *perm, cudaStream_t st);
// tensor-core path (ile_tc.cu)
int ile_tc_kpad(int prec, int M);
int ile_tc_tpad(int T_ext);
size_t ile_tc_q_bytes(int prec, int K, int M, int T_ext);
// Columns appended to every detector's operand rows for the quadratic term (ile_tc.cu): the real
// form of U_k and V_k, so that one extra MMA per detector gives U_k c and V_k c.
#define ILE_QCOLS 128
// The fused kernel's quadratic-term job reads the block packed into the first ILE_QUAD_NCOL of
// those columns: four blocks of 24 (column 24 (b % 4) + 4 (b / 4) + p; 24 = 4 ceil(ILE_MAX_MODES / 4)).
#define ILE_QUAD_NCOL 96
static_assert(4 * ((ILE_MAX_MODES + 3) / 4) <= ILE_QUAD_NCOL / 4, "quadratic-term blocks");
// quad: [K][KPq][ILE_QCOLS] FP32 real-form block, KPq the BF16X3 operand rows (may be null)
// Qp (FP32 [K][2M][T]) from the device copy of the caller's Q (FP64 complex [K][M][T]); ILE_FLAG_NONFINITE in
// *chk for a non-finite entry
cudaError_t ile_launch_q_convert(const double2 *Q64, int K, int M, int T, float *Qp, unsigned *chk, cudaStream_t st);
cudaError_t ile_launch_tc_split(int prec, const PointParams &pp, const float *Qp, const float *quad, void *hi,
                                void *lo, cudaStream_t st);
cudaError_t ile_launch_tc(int prec, const PointParams &pp, const void *hi, const void *lo, IleScratch s,
                          const int *perm, int64_t N, double *out, int full_grid, LoudList loud, unsigned *flags,
                          cudaStream_t st);
// full_grid 0: lnL_t into out (caller order); 1: the grid lnL(n, j) into out (caller order);
// 2: the data term D(n, j) in FP32 into grid_f, rows in processing (sorted) order
// (scr, grid mode 2 only, may be null: the per-sample C, I0, W, A are written there too)
cudaError_t ile_launch_tc2(const PointParams &pp, const void *hi, const void *lo, int TP, int KP, const float *UV,
                           const double *samples, const int *perm, int64_t N, double *out, float *grid_f,
                           int full_grid, LoudList loud, unsigned *flags, cudaStream_t st,
                           const IleScratch *scr = nullptr);
// the same kernel in TF32x3 with its A operand in TMEM (ile_tc3.cu), for points with
// ile_tc3_fits(K, KP) (KP the TF32 operand rows); full_grid 0 or 1
bool ile_tc3_fits(int K, int KP);
cudaError_t ile_launch_tc3(const PointParams &pp, const void *hi, const void *lo, int TP, int KP,
                           const double *samples, const int *perm, int64_t N, double *out, int full_grid,
                           LoudList loud, unsigned *flags, cudaStream_t st);
// adjoint (ile_adjoint.cu)
int ile_grad_q_splits(const PointParams &pp, int64_t N, int n_sm);
int ile_grad_uv_blocks(int64_t N, int n_sm);
// Din: the data term D(n, j) in processing order (from ile_launch_tc2, grid mode 2), or NULL to
// recompute it on CUDA cores.  With Din and the transposed split operand QThi / QTlo (from
// ile_launch_grad_qt) and ile_grad_tc_ok(pp), the E and slope contraction runs on the tensor
// cores; a bounded wait that runs out sets ILE_FLAG_TIMEOUT in *flags.
bool ile_grad_tc_ok(const PointParams &pp);
size_t ile_grad_qt_bytes(const PointParams &pp);
cudaError_t ile_launch_grad_qt(const PointParams &pp, const float *Qp, void *hi, void *lo, cudaStream_t st);
cudaError_t ile_launch_grad_main(const PointParams &pp, const float *Qp, const float *UV, IleScratch s,
                                 const int *perm, const double *samples, const double *g_lnL, int64_t N, float *pig,
                                 const float *Din, const void *QThi, const void *QTlo, unsigned *flags,
                                 double *g_samples, double *lnl_out, cudaStream_t st);
// tc: the sample-reduction GEMM on the tensor cores (BF16x3 split operands; bounded waits report
// through ILE_FLAG_TIMEOUT in *flags), else FP32 on CUDA cores
cudaError_t ile_launch_grad_q(const PointParams &pp, const float *pig, IleScratch s, int64_t N, int nsplit,
                              float *part, double *gQ, bool tc, unsigned *flags, cudaStream_t st);
cudaError_t ile_launch_grad_uv(const PointParams &pp, const double *samples, const double *g_lnL, int64_t N, int nblk,
                               float *part, double *gU, double *gV, cudaStream_t st);
// g_n = scale * d ln L_marg / d lnL_t(n) = scale * exp(ln w_n - max) / S1, from the result of
// ile_launch_mc (ile_mc.cu); scale = *scale_dev when scale_dev is not null
cudaError_t ile_launch_mc_weights(const double *lnL_t, const double *ln_prior, const double *ln_ps, int64_t N,
                                  const double *result, const double *scale_dev, double scale, double *g,
                                  cudaStream_t st);
// batched adaptive-run kernels (per-point state arrays indexed by point: cdf [P][7][101],
// lnps [P][7][100], hist_fx / hist [P][7][100], pooled [P][4], iter_log [P][64][2], iter [P],
// iter_res [P][8]); blk256 / hblk: (point, first sample) of each 256-sample / hist-chunk block
int ile_hist_chunk();
cudaError_t ile_launch_batch_reset(int n_points, const IleBatchPoint *bp, uint64_t *cdf, float *lnps_tab,
                                   double *pooled, int *iter_dev, unsigned long long *hist_fx, double *hist,
                                   double *iter_log, cudaStream_t st);
cudaError_t ile_launch_batch_sample(const IleBatchPoint *bp, const int2 *blk256, int n_blk, const uint64_t *cdf,
                                    const float *lnps_tab, const int *iter_dev, double *theta, double *lnw_prior,
                                    uint8_t *bins, cudaStream_t st);
cudaError_t ile_launch_batch_adapt(int n_points, const IleBatchPoint *bp, const int2 *hblk, int n_hblk,
                                   const double *lnL, const double *lnw_prior, const uint8_t *bins,
                                   const double *iter_res, unsigned long long *hist_fx, double *hist, uint64_t *cdf,
                                   float *lnps_tab, double *pooled, double *iter_log, int *iter_dev,
                                   cudaStream_t st);
cudaError_t ile_launch_batch_sort(int n_points, const IleBatchPoint *bp, const int2 *blk256, int n_blk,
                                  const double *theta, int *keys, int *buckets, int *perm, cudaStream_t st);
int ile_mc_chunk();
cudaError_t ile_launch_batch_mc(int n_points, const IleBatchPoint *bp, const int2 *mblk, int n_mblk,
                                const int *mblk_first, const double *lnL, const double *lnw_prior, double *partials,
                                double *iter_res, cudaStream_t st);
// batched fused kernel: items are (point, tile) pairs; LK, LM, LKP the largest sizes of the batch
int ile_tc2_tile();
// a_tmem: 0 = A operand in shared memory, 1 = in TMEM (wider windows; see ile_tc2.cu)
size_t ile_tc2_batch_smem(int a_tmem, int LK, int LM, int LKP, int NB);
bool ile_tc2_batch_fits(int a_tmem, int LK, int LM, int LKP, int NB);
// admissible window widths [lo, hi] of a placement; returns the default width
int ile_tc2_nwcol_range(int a_tmem, int *lo, int *hi);
cudaError_t ile_launch_tc2_batch(const Tc2Point *pts_dev, const int2 *items_dev, int64_t nitems, int LK, int LM,
                                 int LKP, int a_tmem, int NB, int nwcol, int grid, unsigned *flags, cudaStream_t st);
cudaError_t ile_launch_mc(const double *lnL_t, const double *ln_prior, const double *ln_ps, int64_t N,
                          double *partials, int n_part, double *result, cudaStream_t st);
int ile_mc_partial_count(int64_t N);
int ile_hist_partial_count(int64_t N);
cudaError_t ile_launch_sampler_reset(const IleSamplerParams &sp, uint64_t *cdf, float *lnps_tab, double *pooled,
                                     int *iter_dev, int iter0, cudaStream_t st);
cudaError_t ile_launch_lnps(const IleSamplerParams &sp, const uint64_t *cdf, float *lnps_tab, cudaStream_t st);
// gmm_tab: [7] sampler tables (used for the dimensions in sp.gmm_mask; may be NULL when it is 0);
// u_gmm: [n_gmm][N] sampling variables of the mixture dimensions, in ascending dimension order
// pair_tab / u_pair: the sky pair's table and the sampling variables of the pair [2][N] (used when
// sp.gmm_pair; may be NULL otherwise); a pair draw that finds no point of the rectangle in 1024
// attempts sets ILE_FLAG_RANGE in *flags
cudaError_t ile_launch_sample(const IleSamplerParams &sp, const uint64_t *cdf, const float *lnps_tab,
                              const IleGmmTab *gmm_tab, const IleGmm2Tab *pair_tab, const int *iter_dev, int64_t N,
                              double *theta, double *lnw_prior, uint8_t *bins, float *u_gmm, float *u_pair,
                              unsigned *flags, cudaStream_t st);
// the sky pair's mixture (ile_gmm.cu): table from cur; em_iters EM steps and the merge of the
// iteration's pair samples u_pair [2][N] (part: ile_gmm2_part_doubles() doubles)
size_t ile_gmm2_part_doubles();
cudaError_t ile_launch_gmm2_table(const IleGmm2 *cur, IleGmm2Tab *tab, cudaStream_t st);
cudaError_t ile_launch_gmm2_update(const float *u_pair, const double *lnL, const double *lnw_prior,
                                   const double *iter_res, int64_t N, int em_iters, IleGmm2 *cur, IleGmm2 *bat,
                                   IleGmm2Tab *tab, double *part, cudaStream_t st);
// the initial pair model (host; ile_gmm.cu): C components on the rectangle's diagonal
void ile_gmm2_init(IleGmm2 &g, int C, const double lo[2], const double hi[2]);
// Bounded-wait check (ile_selftest.cu): one block waits on an mbarrier phase nothing completes, for
// about timeout_s, with the kernels' bounded sleeping wait; it then sets ILE_FLAG_TIMEOUT.
cudaError_t ile_launch_wait_check(unsigned *flags, double timeout_s, cudaStream_t st);
// Gaussian-mixture adaptation (ile_gmm.cu).  cur, bat, tab: [7] on the device; part: scratch of
// ile_gmm_part_doubles() doubles.  ile_launch_gmm_table rebuilds tab from cur for the dimensions
// in mask; ile_launch_gmm_update runs em_iters EM steps and the merge (cur updated, N samples).
size_t ile_gmm_part_doubles();
cudaError_t ile_launch_gmm_table(unsigned mask, const IleGmm *cur, IleGmmTab *tab, cudaStream_t st);
cudaError_t ile_launch_gmm_update(unsigned mask, const float *u_gmm, const double *lnL, const double *lnw_prior,
                                  const double *iter_res, int64_t N, int em_iters, IleGmm *cur, IleGmm *bat,
                                  IleGmmTab *tab, double *part, cudaStream_t st);
cudaError_t ile_launch_adapt(const double *lnL, const double *lnw_prior, const uint8_t *bins, int64_t N,
                             const double *iter_res, const IleSamplerParams &sp, double eps,
                             unsigned long long *hist_fx, double *hist, uint64_t *cdf, float *lnps_tab, double *pooled,
                             double *iter_log, int *iter_dev, int update_tables, cudaStream_t st);

// distance-marginalisation tables (ile_dmarg.cu): fills dm (on = 1) and the device tables in `buf`
// (ile_dmarg_buffer_bytes() bytes, 256-byte aligned); synchronous
size_t ile_dmarg_buffer_bytes();
cudaError_t ile_build_dmarg(double d_min, double d_max, double d_ref, void *buf, DmargParams &dm, cudaStream_t st);
cudaError_t ile_launch_dmarg_eval(const DmargParams &dm, const double *a, const double *b, int64_t n, double *out,
                                  cudaStream_t st);

// inner-product arrays of Eq. (eq:QUV) from modes, PSDs and data (ile_quv.cu); z: scratch of
// K * M * L complex doubles
cudaError_t ile_launch_quv(int K, int M, int64_t L, const double *h, const double *psd, const double *d, double df,
                           double f_low, double t_start, double fs, int T_ext, double *z, double *Q, double *U,
                           double *V, cudaStream_t st);

// ------------------------------------------------------------------ host helpers (ile_api.cu)
ile_status ile_prepare_point(int n_det, int n_modes, const int *lm, const double *det_tensor,
                             const double *det_pos_m, const double *Q, int T_ext, double t_start_s, double fs_hz,
                             const double *U, const double *V, int n_window, double gmst_rad, double d_ref_mpc,
                             PointParams &pp_out, std::vector<float> &qp, std::vector<float> &uv,
                             std::vector<float> &quad, bool host_q = true);
void ile_fill_result(const double pooled[4], const double *ilog, int n_iter, ile_adapt_result *out);
