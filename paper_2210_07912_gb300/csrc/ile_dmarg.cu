// ile_dmarg.cu -- distance marginalisation (App. "Distance marginalization"; the integral is
// written out in ile_internal.cuh): the two lookup tables of ln F(a, b), built in FP64 on the
// device, one thread per entry, when ile_set_distance_marginalization is called.
//
// For an entry (a, b), with u = a / 2b: the integrand C x^-4 exp(a x - b x^2 - E*) on
// [x_min, x_max] (x = D_ref / D; C x^-4 dx is the D^2 prior; E* the largest value of a x - b x^2
// on the range, at x* = clip(u)) is at most 1 at x*; its width there is l = 1/sqrt(2b) for an
// interior x* and min(1/sqrt(2b), 1/(2b |u - x*|)) at an end.  The window [x* - 40 l, x* + 40 l]
// (clipped to the range; the whole range when l is large) is integrated with 32 panels of the
// 8-point Gauss-Legendre rule.  Where the prior's x^-4 growth towards x_min competes with the
// likelihood peak (the integrand is then bimodal), l is large and the window is the whole range.
// Why two tables: ln F is a cumulant-generating function in a (second derivative
// = variance of x <= 0.2), so for small and moderate b it is smooth on an (a, b) grid, while for
// large b the peak is narrow and is resolved in standardised coordinates near the range ends.
#include <math.h>

#include <vector>

#include "ile_internal.cuh"

namespace {

// table 1 (b < B_SPLIT): ln F on a = A0 sinh(tau) x b = exp(s)
constexpr double B_SPLIT = 10.0;
constexpr double A0 = 2.0;
constexpr double A1_MAX = 2e4;     // |a| covered
constexpr double DTAU1 = 0.01;
constexpr double S1_LO = -13.815510557964274;  // ln 1e-6
constexpr double DS1 = 0.01;
// table 2 (b >= B_SPLIT): H = ln F - E* on tau(u) x s = ln b
constexpr double EPS2 = 0.005;
constexpr double Z2_MAX = 1e5;     // |u - x_c| / w_z covered
constexpr double DTAU2 = 0.02;
constexpr double S2_HI = 13.815510557964274;   // ln 1e6
constexpr double DS2 = 0.01;

struct Gl8 {
    double x[8], w[8];
};

// 8-point Gauss-Legendre nodes and weights on [-1, 1]: Newton iteration on P_8 (textbook
// construction).
Gl8 gauss_legendre8() {
    Gl8 g;
    const int n = 8;
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 60; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        g.x[i] = z;
        g.w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return g;
}

struct Range {
    double xmin, xmax, cnorm;
};

// ln F(a, b) - E*(a, b), and E*, in FP64.
__device__ double lnF_minus_estar(const Gl8 &gl, const Range &r, double a, double b, double *estar_out) {
    const double u = a / (2.0 * b);
    const double xs = fmin(fmax(u, r.xmin), r.xmax);
    const double estar = a * xs - b * xs * xs;
    const double sigma = 1.0 / sqrt(2.0 * b);
    const double slope = 2.0 * b * fabs(u - xs);
    const double ell = slope > 0.0 ? fmin(sigma, 1.0 / slope) : sigma;
    // outside the window the exponent is below -40 relative to x*, which the prior's x^-4 (at
    // most 10^4 over the range) cannot make up
    const double L = fmax(r.xmin, xs - 40.0 * ell), Hh = fmin(r.xmax, xs + 40.0 * ell);
    const int panels = 32;
    const double h = (Hh - L) / panels;
    double sum = 0.0;
    for (int p = 0; p < panels; p++) {
        const double c = L + (p + 0.5) * h;
        for (int q = 0; q < 8; q++) {
            const double x = c + 0.5 * h * gl.x[q];
            const double x2 = x * x;
            sum += 0.5 * h * gl.w[q] * r.cnorm / (x2 * x2) * exp(a * x - b * x2 - estar);
        }
    }
    *estar_out = estar;
    return log(sum);
}

__global__ void table1_kernel(Gl8 gl, Range r, const double *__restrict__ a_nodes, int n1a, int n1s,
                              float *__restrict__ t1) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n1a * n1s) return;
    const int k = idx / n1a, i = idx % n1a;
    const double b = exp(S1_LO + k * DS1);
    double estar;
    const double h = lnF_minus_estar(gl, r, a_nodes[i], b, &estar);
    t1[idx] = (float)(h + estar);
}

__global__ void table2_kernel(Gl8 gl, Range r, const double *__restrict__ u_nodes, int n2t, int n2s, double s2_lo,
                              float *__restrict__ t2) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n2t * n2s) return;
    const int k = idx / n2t, i = idx % n2t;
    const double b = exp(s2_lo + k * DS2);
    double estar;
    t2[idx] = (float)lnF_minus_estar(gl, r, 2.0 * b * u_nodes[i], b, &estar);
}

struct Layout {
    int n1a, n1s, n2t, n2s;
    double tau1_max, tau2_lo, tau2_hi, s2_lo;
    size_t off_t1, off_a1, off_t2, off_t1p, off_t2p, off_scratch, bytes;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout() {
    Layout L{};
    L.tau1_max = asinh(A1_MAX / A0);
    L.n1a = (int)ceil(2.0 * L.tau1_max / DTAU1) + 1;
    L.n1s = (int)ceil((log(B_SPLIT) - S1_LO) / DS1) + 2;
    L.s2_lo = log(B_SPLIT);
    L.n2s = (int)ceil((S2_HI - L.s2_lo) / DS2) + 1;
    // tau2 range for |u - x_c| <= Z2_MAX w_z: independent of the distance range's scale only
    // through eps; the node count is fixed by the worst case x_min -> 0, x_max -> 1.
    L.n2t = 4096;
    L.off_t1 = 0;
    L.off_a1 = align256(L.off_t1 + sizeof(float) * (size_t)L.n1a * L.n1s);
    L.off_t2 = align256(L.off_a1 + sizeof(float2) * (size_t)L.n1a);
    L.off_t1p = align256(L.off_t2 + sizeof(float) * (size_t)L.n2t * L.n2s);
    L.off_t2p = align256(L.off_t1p + sizeof(float2) * (size_t)L.n1a * L.n1s);
    L.off_scratch = align256(L.off_t2p + sizeof(float2) * (size_t)L.n2t * L.n2s);
    L.bytes = align256(L.off_scratch + sizeof(double) * (size_t)(L.n1a > L.n2t ? L.n1a : L.n2t));
    return L;
}

double tau2_of(double u, double xmin, double xmax) { return asinh((u - xmin) / EPS2) + asinh((u - xmax) / EPS2); }

// Node pairs (t[i], t[i + 1]) of a row-major table with ncol columns, so that one 8-byte load
// gives both ends of an interpolation interval (the last column pairs with itself; the lookups
// never start an interval there).
__global__ void pair_kernel(const float *__restrict__ t, int ncol, int64_t n, float2 *__restrict__ tp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % ncol);
    tp[i] = make_float2(t[i], c + 1 < ncol ? t[i + 1] : t[i]);
}

__global__ void dmarg_eval_kernel(const DmargParams dm, const double *__restrict__ a, const double *__restrict__ b,
                                  int64_t n, double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DmargSample q = ile_dmarg_sample(dm, (float)b[i]);
    out[i] = (double)ile_dmarg_lnF(dm, q, (float)a[i]);
}

}  // namespace

size_t ile_dmarg_buffer_bytes() { return layout().bytes; }

cudaError_t ile_launch_dmarg_eval(const DmargParams &dm, const double *a, const double *b, int64_t n, double *out,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    dmarg_eval_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dm, a, b, n, out);
    return cudaGetLastError();
}

cudaError_t ile_build_dmarg(double d_min, double d_max, double d_ref, void *buf, DmargParams &dm, cudaStream_t st) {
    const Layout L = layout();
    Range r;
    r.xmin = d_ref / d_max;
    r.xmax = d_ref / d_min;
    r.cnorm = 3.0 * d_ref * d_ref * d_ref / (d_max * d_max * d_max - d_min * d_min * d_min);
    const double xc = 0.5 * (r.xmin + r.xmax), wz = 0.125 * (r.xmax - r.xmin);
    uint8_t *base = static_cast<uint8_t *>(buf);
    float *t1 = reinterpret_cast<float *>(base + L.off_t1);
    float2 *a1 = reinterpret_cast<float2 *>(base + L.off_a1);
    float *t2 = reinterpret_cast<float *>(base + L.off_t2);
    float2 *t1p = reinterpret_cast<float2 *>(base + L.off_t1p);
    float2 *t2p = reinterpret_cast<float2 *>(base + L.off_t2p);
    double *nodes = reinterpret_cast<double *>(base + L.off_scratch);
    const Gl8 gl = gauss_legendre8();
    // table 1 nodes
    std::vector<double> an(L.n1a);
    std::vector<float2> anf(L.n1a);  // (a_i, 1 / (a_{i+1} - a_i)) for the per-bin lerp weight
    const double dtau1 = 2.0 * L.tau1_max / (L.n1a - 1);
    for (int i = 0; i < L.n1a; i++) an[i] = A0 * sinh(-L.tau1_max + i * dtau1);
    for (int i = 0; i < L.n1a; i++)
        anf[i] = make_float2((float)an[i], i + 1 < L.n1a ? (float)(1.0 / (an[i + 1] - an[i])) : 0.f);
    cudaError_t e = cudaMemcpyAsync(nodes, an.data(), sizeof(double) * L.n1a, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a1, anf.data(), sizeof(float2) * L.n1a, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    table1_kernel<<<(L.n1a * L.n1s + 127) / 128, 128, 0, st>>>(gl, r, nodes, L.n1a, L.n1s, t1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the node scratch is reused below
    if (e != cudaSuccess) return e;
    // table 2 nodes: u_i with tau2(u_i) uniform (tau2 is increasing in u; bisection)
    const double ulo = xc - Z2_MAX * wz, uhi = xc + Z2_MAX * wz;
    const double tlo = tau2_of(ulo, r.xmin, r.xmax), thi = tau2_of(uhi, r.xmin, r.xmax);
    const double dtau2 = (thi - tlo) / (L.n2t - 1);
    std::vector<double> un(L.n2t);
    for (int i = 0; i < L.n2t; i++) {
        const double t = tlo + i * dtau2;
        double lo = ulo, hi = uhi;
        for (int it = 0; it < 200; it++) {
            const double m = 0.5 * (lo + hi);
            if (tau2_of(m, r.xmin, r.xmax) < t) lo = m; else hi = m;
        }
        un[i] = 0.5 * (lo + hi);
    }
    e = cudaMemcpyAsync(nodes, un.data(), sizeof(double) * L.n2t, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    table2_kernel<<<(L.n2t * L.n2s + 127) / 128, 128, 0, st>>>(gl, r, nodes, L.n2t, L.n2s, L.s2_lo, t2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        const int64_t n1 = (int64_t)L.n1a * L.n1s, n2 = (int64_t)L.n2t * L.n2s;
        pair_kernel<<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(t1, L.n1a, n1, t1p);
        pair_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(t2, L.n2t, n2, t2p);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    dm = DmargParams{};
    dm.on = 1;
    dm.xmin = (float)r.xmin;
    dm.xmax = (float)r.xmax;
    dm.b_split = (float)B_SPLIT;
    dm.n1a = L.n1a;
    dm.n1s = L.n1s;
    dm.A0 = (float)A0;
    dm.inv_A0 = (float)(1.0 / A0);
    dm.tau1_max = (float)L.tau1_max;
    dm.inv_dtau1 = (float)(1.0 / dtau1);
    dm.s1_lo = (float)S1_LO;
    dm.ds1 = (float)DS1;
    dm.t1 = t1;
    dm.a1 = a1;
    dm.n2t = L.n2t;
    dm.n2s = L.n2s;
    dm.eps = (float)EPS2;
    dm.inv_eps = (float)(1.0 / EPS2);
    dm.tau2_lo = (float)tlo;
    dm.inv_dtau2 = (float)(1.0 / dtau2);
    dm.s2_lo = (float)L.s2_lo;
    dm.inv_ds2 = (float)(1.0 / DS2);
    dm.t2 = t2;
    dm.t1p = t1p;
    dm.t2p = t2p;
    return cudaSuccess;
}
