// ile_api.cu -- host side of the libile C ABI (include/ile.h): context, argument checks, data
// upload and the launch sequence of each entry point.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <unordered_map>
#include <vector>

#include "ile_internal.cuh"

struct ile_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    ile_prec prec = ILE_PREC_FP32;
    bool has_data = false;
    PointParams pp{};
    // point data
    double2 *Q64 = nullptr, *U64 = nullptr, *V64 = nullptr;  // FP64 copies for the refinement (ile_refine.cu)
    Refine64 r64{};
    int *loud = nullptr;   // [2 cap + 1] loud samples of the last evaluation (count, then (0, index) pairs)
    bool refine = true;    // refine loud samples in FP64 (ile_set_refine)
    float *Qp = nullptr;   // [K][2M][T_ext]
    float *UV = nullptr;   // [K][P][4]
    float *Qquad = nullptr;  // [K][KP][ILE_QCOLS] real form of U, V (quadratic-term MMA operand)
    void *dm_table = nullptr;  // distance-marginalisation tables (ile_dmarg.cu)
    // tensor-core operand rows (hi, lo) of the current point, per split precision (ile_tc.cu)
    void *Qtc[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    bool Qtc_ready[3] = {false, false, false};
    size_t Qtc_bytes[3] = {0, 0, 0};
    // transposed split operand (hi, lo) of the adjoint's tensor-core E contraction (ile_adjoint.cu)
    void *Qadj[2] = {nullptr, nullptr};
    bool Qadj_ready = false;
    size_t Qadj_bytes = 0;
    // delay-sort scratch
    int *keys = nullptr, *buckets = nullptr, *perm = nullptr;
    // per-sample scratch
    int64_t cap = 0;
    IleScratch s{};
    double *theta = nullptr;  // staged host samples [7][cap]
    double *out = nullptr;    // [cap] (or grid)
    size_t out_bytes = 0;
    double *lnp = nullptr, *lnps = nullptr;
    double *part = nullptr;
    int part_cap = 0;
    double *result = nullptr;  // [8]
    unsigned *flags = nullptr;
    char err[256] = {0};
    // adaptive integrator state (ile_adapt.cu)
    bool adapt_ready = false;
    IleSamplerParams sp{};
    double eps = 0.1;
    int64_t adapt_N = 0;
    uint64_t *a_cdf = nullptr;
    float *a_lnps = nullptr;
    double *a_hist = nullptr;
    unsigned long long *a_hist_fx = nullptr;
    double *a_pooled = nullptr, *a_iter_log = nullptr, *a_iter_res = nullptr, *a_lnwp = nullptr, *a_lnl = nullptr;
    int *a_iter = nullptr;
    uint8_t *a_bins = nullptr;
    int64_t a_cap = 0;
    // Gaussian-mixture dimensions (ile_gmm.cu)
    int gmm_iters = 0;
    IleGmm *g_cur = nullptr, *g_bat = nullptr;
    IleGmmTab *g_tab = nullptr;
    double *g_part = nullptr;
    float *a_u = nullptr;  // [n mixture dims][N]
    // the sky pair's correlated mixture (ile_gmm.cu)
    IleGmm2 *g2_cur = nullptr, *g2_bat = nullptr;
    IleGmm2Tab *g2_tab = nullptr;
    double *g2_part = nullptr;
    float *a_upair = nullptr;  // [2][N]
    int64_t a_upair_cap = 0;
    size_t a_u_bytes = 0;
    // adjoint scratch (ile_adjoint.cu)
    float *pig = nullptr;      // [N][N_t] g_n * pi(n, j)
    size_t pig_bytes = 0;
    float *gq_part = nullptr;  // [splits][K][2M][T_ext]
    size_t gq_bytes = 0;
    float *guv_part = nullptr; // [blocks][K][P][4]
    size_t guv_bytes = 0;
    int *ss_work = nullptr;    // the stable sort's key, index and histogram arrays
    size_t ss_bytes = 0;
    double *g_in = nullptr;    // staged host upstream gradient [cap]
    double *g_out = nullptr;   // staged g_theta [7][cap] and g_Q, g_U, g_V for host-pointer calls
    size_t g_out_bytes = 0;
    int n_sm = 0;
    // device memory owned by the context (ctx_malloc / ctx_free) and its optional cap
    size_t mem_limit = 0, mem_used = 0;
    std::unordered_map<void *, size_t> allocs;
    // stage timing
    bool profiling = false;
    std::vector<cudaEvent_t> ev[ILE_NSTAGE];
    size_t ev_used[ILE_NSTAGE] = {0};
    int64_t kernels[ILE_NSTAGE] = {0};
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

ile_status cuda_fail(ile_ctx *c, cudaError_t e, const char *where) {
    if (c) snprintf(c->err, sizeof c->err, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ILE_E_NOMEM : ILE_E_CUDA;
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

// Device allocations of a context go through ctx_malloc / ctx_free, which keep the bytes in use
// so that ile_set_memory_limit can refuse an allocation (ILE_E_NOMEM) before cudaMalloc is called.
cudaError_t ctx_malloc(ile_ctx *ctx, void **p, size_t bytes) {
    if (ctx->mem_limit && ctx->mem_used + bytes > ctx->mem_limit) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        ctx->mem_used += bytes;
        ctx->allocs[*p] = bytes;
    }
    return e;
}

void ctx_free(ile_ctx *ctx, void *p) {
    if (!p) return;
    const auto it = ctx->allocs.find(p);
    if (it != ctx->allocs.end()) {
        ctx->mem_used -= it->second;
        ctx->allocs.erase(it);
    }
    cudaFree(p);
}

template <typename T>
cudaError_t grow(ile_ctx *ctx, T **p, size_t bytes) {
    ctx_free(ctx, *p);
    *p = nullptr;
    return ctx_malloc(ctx, (void **)p, bytes);
}

// Keep *p when its allocation already holds `bytes` (a point's arrays are re-used by the next
// point of the same or a smaller shape: no cudaFree / cudaMalloc per ile_set_data), else grow.
template <typename T>
cudaError_t reserve(ile_ctx *ctx, T **p, size_t bytes) {
    if (*p) {
        const auto it = ctx->allocs.find((void *)*p);
        if (it != ctx->allocs.end() && it->second >= bytes) return cudaSuccess;
    }
    return grow(ctx, p, bytes);
}

// Bracket one launch of stage `stage` with events on the context stream (when profiling) and
// with an NVTX range on the host timeline (a no-op unless a tool such as Nsight is attached).
const char *const kStageName[ILE_NSTAGE] = {"ile:sample", "ile:coefficients", "ile:contraction",
                                            "ile:mc_reduce", "ile:adapt",  "ile:adjoint", "ile:refine"};
struct StageScope {
    ile_ctx *c;
    int stage;
    StageScope(ile_ctx *ctx, int s, int n_kernels = 1) : c(ctx), stage(s) {
        nvtxRangePushA(kStageName[s]);
        if (c->profiling) c->kernels[s] += n_kernels;
        mark();
    }
    ~StageScope() {
        mark();
        nvtxRangePop();
    }
    void mark() {
        if (!c->profiling) return;
        auto &v = c->ev[stage];
        if (c->ev_used[stage] == v.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            v.push_back(e);
        }
        cudaEventRecord(v[c->ev_used[stage]++], c->stream);
    }
};

ile_status ensure_samples(ile_ctx *ctx, int64_t N) {
    if (N <= ctx->cap) return ILE_OK;
    const int K = ctx->pp.K, R = 2 * ctx->pp.M;
    int64_t cap = N;
    // until every buffer below is in place the scratch counts as empty (a failed growth, e.g. past
    // the memory cap, leaves some of them released)
    ctx->cap = 0;
    ctx->part_cap = 0;
    CK(grow(ctx, &ctx->s.C, sizeof(float) * (size_t)ILE_MAX_DET * 2 * ILE_MAX_MODES * cap));
    CK(grow(ctx, &ctx->s.I0, sizeof(int) * (size_t)ILE_MAX_DET * cap));
    CK(grow(ctx, &ctx->s.W, sizeof(float) * (size_t)ILE_MAX_DET * cap));
    CK(grow(ctx, &ctx->s.A, sizeof(float) * (size_t)cap));
    CK(grow(ctx, &ctx->theta, sizeof(double) * ILE_NDIM * (size_t)cap));
    CK(grow(ctx, &ctx->lnp, sizeof(double) * (size_t)cap));
    CK(grow(ctx, &ctx->lnps, sizeof(double) * (size_t)cap));
    CK(grow(ctx, &ctx->keys, sizeof(int) * (size_t)cap));
    CK(grow(ctx, &ctx->perm, sizeof(int) * (size_t)cap));
    CK(grow(ctx, &ctx->g_in, sizeof(double) * (size_t)cap));
    CK(grow(ctx, &ctx->loud, sizeof(int) * (size_t)(2 * cap + 1)));
    if (!ctx->buckets) CK(ctx_malloc(ctx, (void **)&ctx->buckets, sizeof(int) * ile_sort_key_buckets()));
    int np = ile_mc_partial_count(cap);
    CK(grow(ctx, &ctx->part, sizeof(double) * 3 * (size_t)np));
    ctx->part_cap = np;
    (void)K;
    (void)R;
    ctx->cap = cap;
    return ILE_OK;
}

ile_status ensure_out(ile_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->out_bytes) return ILE_OK;
    ctx->out_bytes = 0;
    CK(grow(ctx, &ctx->out, bytes));
    ctx->out_bytes = bytes;
    return ILE_OK;
}

double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; i++) f *= i;
    return f;
}

// Polynomial form of d^l_{m,2}(iota) in c = cos(iota/2), s = sin(iota/2) (Wigner's formula).
// Terms of d^l_{m,2}(iota) = sum_t coef_t cos(iota/2)^p_t sin(iota/2)^q_t (the explicit Wigner
// small-d sum) and the normalisation sqrt((2l+1)/4pi) of _{-2}Y_lm, in FP64.
bool wigner_terms64(int l, int m, Mode64 &md) {
    md.l = l;
    md.m = m;
    md.norm = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
    md.nterms = 0;
    const double root = sqrt(factorial(l + m) * factorial(l - m) * factorial(l + 2) * factorial(l - 2));
    for (int sp = 0; sp <= 2 * l; sp++) {  // sp = power of s = 2k - 2 + m
        int twok = sp + 2 - m;
        if (twok < 0 || (twok & 1)) continue;
        int k = twok / 2;
        int f1 = l + 2 - k, f2 = l - m - k, f3 = k + m - 2;
        if (f1 < 0 || f2 < 0 || f3 < 0) continue;
        if (md.nterms >= 4) return false;
        double sign = (f3 % 2 == 0) ? 1.0 : -1.0;
        md.coef[md.nterms] = sign * root / (factorial(f1) * factorial(k) * factorial(f2) * factorial(f3));
        md.p[md.nterms] = 2 * l - sp;
        md.q[md.nterms] = sp;
        md.nterms++;
    }
    return true;
}

bool wigner_terms(int l, int m, ModeTab &md) {
    Mode64 d;
    if (!wigner_terms64(l, m, d)) return false;
    md.l = l;
    md.m = m;
    md.norm = (float)d.norm;
    md.nterms = d.nterms;
    for (int t = 0; t < d.nterms; t++) {
        md.t[t].coef = (float)d.coef[t];
        md.t[t].p = d.p[t];
        md.t[t].q = d.q[t];
    }
    return true;
}

bool finite_array(const double *p, size_t n) {
    for (size_t i = 0; i < n; i++)
        if (!isfinite(p[i])) return false;
    return true;
}

ile_status read_flags(ile_ctx *ctx) {
    unsigned f = 0;
    CK(cudaMemcpyAsync(&f, ctx->flags, sizeof f, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (f) CK(cudaMemsetAsync(ctx->flags, 0, sizeof(unsigned), ctx->stream));
    if (f & ILE_FLAG_TIMEOUT) return ILE_E_TIMEOUT;
    if (f & ILE_FLAG_RANGE) return ILE_E_RANGE;
    if (f & ILE_FLAG_NONFINITE) return ILE_E_NONFINITE;
    return ILE_OK;
}

// Host-pointer calls: the device-side flags are read (and the stream synchronised) before any
// output is copied back, so a call that fails leaves the caller's buffers untouched.
ile_status finish_host_copies(ile_ctx *ctx) {
    CK(cudaStreamSynchronize(ctx->stream));
    return ILE_OK;
}

// Operand rows of the split-precision contraction for the current point (built once per point).
ile_status ensure_tc_operands(ile_ctx *ctx, int prec) {
    if (ctx->Qtc_ready[prec]) return ILE_OK;
    const size_t bytes = ile_tc_q_bytes(prec, ctx->pp.K, ctx->pp.M, ctx->pp.T_ext);
    if (bytes > ctx->Qtc_bytes[prec]) {
        ctx->Qtc_bytes[prec] = 0;
        CK(grow(ctx, &ctx->Qtc[prec][0], bytes));
        CK(grow(ctx, &ctx->Qtc[prec][1], bytes));
        ctx->Qtc_bytes[prec] = bytes;
    }
    CK(ile_launch_tc_split(prec, ctx->pp, ctx->Qp, ctx->Qquad, ctx->Qtc[prec][0], ctx->Qtc[prec][1], ctx->stream));
    ctx->Qtc_ready[prec] = true;
    return ILE_OK;
}

// The adjoint's transposed split operand of the current point (built once per point).
ile_status ensure_adj_operands(ile_ctx *ctx) {
    if (ctx->Qadj_ready) return ILE_OK;
    const size_t bytes = ile_grad_qt_bytes(ctx->pp);
    if (bytes > ctx->Qadj_bytes) {
        ctx->Qadj_bytes = 0;
        CK(grow(ctx, &ctx->Qadj[0], bytes));
        CK(grow(ctx, &ctx->Qadj[1], bytes));
        ctx->Qadj_bytes = bytes;
    }
    CK(ile_launch_grad_qt(ctx->pp, ctx->Qp, ctx->Qadj[0], ctx->Qadj[1], ctx->stream));
    ctx->Qadj_ready = true;
    return ILE_OK;
}

// S1-S5 on device-resident samples; writes lnL_t (or the grid) to dout in the caller's order.
// Samples are first ordered by quantised detector delays (ile_sort.cu) so that a tile of the
// contraction spans few time columns; the per-sample results do not depend on that order.
}  // namespace

// Samples with |max_j D| + A above this go to the FP64 refinement (ile_refine.cu).  The fast paths'
// absolute errors measured against the FP64 oracle on injections of <h0|h0> = 1e2 .. 1e4 stay
// below 1e-6 (FP32, TF32X3) and 5e-6 (BF16X3) of |max_j D| + A, so the samples left to them stay
// below 3e-4.
float ile_refine_threshold(int prec) { return prec == ILE_PREC_BF16X3 ? 50.f : 300.f; }

// FP64 description of a point for the refinement (the arguments have been validated by
// ile_prepare_point).
bool ile_refine_params(int n_det, int n_modes, const int *lm, const double *det_tensor, const double *det_pos_m,
                       int T_ext, double t_start_s, double fs_hz, int n_window, double gmst_rad, double d_ref_mpc,
                       Refine64 &r) {
    r = Refine64{};
    r.K = n_det;
    r.M = n_modes;
    r.Nt = n_window;
    r.T_ext = T_ext;
    r.fs = fs_hz;
    r.t_start = t_start_s;
    r.gmst = gmst_rad;
    r.d_ref = d_ref_mpc;
    r.log_nt = log((double)n_window);
    for (int k = 0; k < n_det; k++) {
        for (int i = 0; i < 9; i++) r.det_tensor[k][i] = det_tensor[9 * k + i];
        for (int i = 0; i < 3; i++) r.det_pos[k][i] = det_pos_m[3 * k + i];
    }
    for (int a = 0; a < n_modes; a++)
        if (!wigner_terms64(lm[2 * a], lm[2 * a + 1], r.mode[a])) return false;
    return true;
}

namespace {

// S1-S5 on device-resident samples; writes lnL_t (or the grid) to dout in the caller's order.
// Samples are first ordered by quantised detector delays (ile_sort.cu) so that a tile of the
// contraction spans few time columns; the per-sample results do not depend on that order.
// lnL_t of loud samples is then recomputed in FP64 (unless the context's refinement is off).
ile_status run_eval(ile_ctx *ctx, const double *dsamples, int64_t N, double *dout, int full_grid,
                    bool nearest = false) {
    ile_status st = ensure_samples(ctx, N);
    if (st != ILE_OK) return st;
    const int prec = (int)ctx->prec;
    PointParams pp = ctx->pp;
    pp.nearest = nearest ? 1 : 0;
    if (prec != ILE_PREC_FP32) {
        st = ensure_tc_operands(ctx, prec);
        if (st != ILE_OK) return st;
    }
    LoudList loud{nullptr, 0.f};
    if (full_grid == 0 && ctx->refine && !pp.dm.on) {
        loud = LoudList{ctx->loud, ile_refine_threshold(prec), 0, ctx->cap};
        CK(cudaMemsetAsync(ctx->loud, 0, sizeof(int), ctx->stream));
    }
    const bool fused = prec == ILE_PREC_BF16X3 ||
                       (prec == ILE_PREC_TF32X3 && ile_tc3_fits(pp.K, ile_tc_kpad(prec, pp.M)));
    if (fused) {
        // fused kernel: S1, S2, S4 are computed inside the tensor-core kernel
        {
            StageScope t(ctx, 1, 3);
            CK(ile_launch_sort(pp, dsamples, N, ctx->keys, ctx->buckets, ctx->perm, ctx->stream));
        }
        StageScope t(ctx, 2);
        if (prec == ILE_PREC_BF16X3)
            CK(ile_launch_tc2(pp, ctx->Qtc[prec][0], ctx->Qtc[prec][1], ile_tc_tpad(pp.T_ext),
                              ile_tc_kpad(prec, pp.M), ctx->UV, dsamples, ctx->perm, N, dout, nullptr, full_grid,
                              loud, ctx->flags, ctx->stream));
        else
            CK(ile_launch_tc3(pp, ctx->Qtc[prec][0], ctx->Qtc[prec][1], ile_tc_tpad(pp.T_ext),
                              ile_tc_kpad(prec, pp.M), dsamples, ctx->perm, N, dout, full_grid, loud, ctx->flags,
                              ctx->stream));
    } else {
        {
            StageScope t(ctx, 1, 4);
            CK(ile_launch_sort(pp, dsamples, N, ctx->keys, ctx->buckets, ctx->perm, ctx->stream));
            CK(ile_launch_prep(pp, ctx->UV, dsamples, ctx->perm, N, ctx->s, ctx->flags, ctx->stream));
        }
        StageScope t(ctx, 2);
        if (prec == ILE_PREC_FP32)
            CK(ile_launch_plain(pp, ctx->Qp, ctx->s, ctx->perm, N, dout, full_grid, loud, ctx->flags,
                                ctx->stream));
        else
            CK(ile_launch_tc(prec, pp, ctx->Qtc[prec][0], ctx->Qtc[prec][1], ctx->s, ctx->perm, N, dout,
                             full_grid, loud, ctx->flags, ctx->stream));
    }
    if (loud.list) {
        StageScope t(ctx, 6);
        Refine64 r = ctx->r64;
        r.thr = loud.thr;
        r.nearest = pp.nearest;
        CK(ile_launch_refine(r, ctx->Q64, ctx->U64, ctx->V64, ctx->Qp, dsamples, N, ctx->loud, ctx->cap, dout,
                             ctx->flags, ctx->n_sm, ctx->stream));
    }
    return ILE_OK;
}

template <typename T>
cudaError_t ensure_bytes(ile_ctx *ctx, T **p, size_t *have, size_t bytes) {
    if (bytes <= *have && *p) return cudaSuccess;
    cudaError_t e = grow(ctx, p, bytes);
    *have = e == cudaSuccess ? bytes : 0;
    return e;
}

// Adjoint of S1-S5 on device-resident arrays (ile_adjoint.cu).  Any of g_theta, gQ, gU, gV, lnl
// may be null.  Samples are delay-sorted first, as in the forward pass.
ile_status run_grad(ile_ctx *ctx, const double *dsamples, const double *dg, int64_t N, double *g_theta, double *gQ,
                    double *gU, double *gV, double *lnl) {
    ile_status st = ensure_samples(ctx, N);
    if (st != ILE_OK) return st;
    const PointParams &pp = ctx->pp;
    if (!ctx->n_sm) CK(cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
    // BF16x3 contexts take the data term D(n, j) from the fused tensor-core kernel (written into
    // the pi buffer, which the adjoint then overwrites with g * pi) instead of recomputing it
    const bool tc2_fwd = ctx->prec == ILE_PREC_BF16X3 && (g_theta || gQ || lnl);
    float *pig = nullptr;
    if (gQ || tc2_fwd) {
        CK(ensure_bytes(ctx, &ctx->pig, &ctx->pig_bytes, sizeof(float) * (size_t)N * pp.Nt));
        pig = ctx->pig;
    }
    // ... and run the E / slope contraction on the tensor cores when it fits shared memory
    const bool tc_adj = tc2_fwd && ile_grad_tc_ok(pp);
    if (tc2_fwd) {
        st = ensure_tc_operands(ctx, ILE_PREC_BF16X3);
        if (st != ILE_OK) return st;
    }
    if (tc_adj) {
        st = ensure_adj_operands(ctx);
        if (st != ILE_OK) return st;
    }
    const int nsplit = ile_grad_q_splits(pp, N, ctx->n_sm);
    const int nblk = ile_grad_uv_blocks(N, ctx->n_sm);
    CK(ensure_bytes(ctx, &ctx->ss_work, &ctx->ss_bytes, sizeof(int) * ile_sort_stable_work_ints(N)));
    if (gQ) CK(ensure_bytes(ctx, &ctx->gq_part, &ctx->gq_bytes, sizeof(float) * (size_t)nsplit * pp.K * 2 * pp.M * pp.T_ext));
    if (gU || gV)
        CK(ensure_bytes(ctx, &ctx->guv_part, &ctx->guv_bytes,
                        sizeof(float) * (size_t)nblk * pp.K * (pp.M * (pp.M + 1) / 2) * 4));
    {
        // (the BF16x3 D(n, j) pass below writes the per-sample coefficients, window placements and
        // quadratic term itself; other contexts form them with the coefficient kernel).  The sort
        // is the stable form: dQ sums over samples in its order, so equal keys keep the caller's
        // order and the call gives the same result on every run.
        StageScope t(ctx, 1, tc2_fwd ? 6 : 7);
        CK(ile_launch_sort_stable(pp, dsamples, N, ctx->keys, ctx->ss_work, ctx->perm, ctx->stream));
        if (!tc2_fwd) CK(ile_launch_prep(pp, ctx->UV, dsamples, ctx->perm, N, ctx->s, ctx->flags, ctx->stream));
    }
    StageScope t(ctx, 5, 1 + (tc2_fwd ? 1 : 0) + (gQ ? 2 : 0) + ((gU || gV) ? 2 : 0));
    if (tc2_fwd)
        CK(ile_launch_tc2(pp, ctx->Qtc[ILE_PREC_BF16X3][0], ctx->Qtc[ILE_PREC_BF16X3][1], ile_tc_tpad(pp.T_ext),
                          ile_tc_kpad(ILE_PREC_BF16X3, pp.M), ctx->UV, dsamples, ctx->perm, N, nullptr, pig, 2,
                          LoudList{nullptr, 0.f, 0, 0}, ctx->flags, ctx->stream, &ctx->s));
    if (g_theta || gQ || lnl)
        CK(ile_launch_grad_main(pp, ctx->Qp, ctx->UV, ctx->s, ctx->perm, dsamples, dg, N, pig,
                                tc2_fwd ? pig : nullptr, tc_adj ? ctx->Qadj[0] : nullptr,
                                tc_adj ? ctx->Qadj[1] : nullptr, ctx->flags, g_theta, lnl, ctx->stream));
    if (gQ)
        CK(ile_launch_grad_q(pp, pig, ctx->s, N, nsplit, ctx->gq_part, gQ, ctx->prec == ILE_PREC_BF16X3, ctx->flags,
                             ctx->stream));
    if (gU || gV) CK(ile_launch_grad_uv(pp, dsamples, dg, N, nblk, ctx->guv_part, gU, gV, ctx->stream));
    return ILE_OK;
}

// Host-pointer wrapper of run_grad: stage inputs, run, copy the requested outputs back.
ile_status run_grad_host(ile_ctx *ctx, const double *samples, const double *g, int64_t N, double *g_theta,
                         double *gQ, double *gU, double *gV, double *lnl) {
    const PointParams &pp = ctx->pp;
    const size_t nth = (size_t)ILE_NDIM * N, nq = 2 * (size_t)pp.K * pp.M * pp.T_ext,
                 nuv = 2 * (size_t)pp.K * pp.M * pp.M;
    CK(ensure_bytes(ctx, &ctx->g_out, &ctx->g_out_bytes, sizeof(double) * (nth + nq + 2 * nuv + (size_t)N)));
    double *d_th = ctx->g_out, *d_q = d_th + nth, *d_u = d_q + nq, *d_v = d_u + nuv, *d_l = d_v + nuv;
    CK(cudaMemcpyAsync(ctx->theta, samples, sizeof(double) * nth, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->g_in, g, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream));
    ile_status st = run_grad(ctx, ctx->theta, ctx->g_in, N, g_theta ? d_th : nullptr, gQ ? d_q : nullptr,
                             gU ? d_u : nullptr, gV ? d_v : nullptr, lnl ? d_l : nullptr);
    if (st != ILE_OK) return st;
    st = read_flags(ctx);
    if (st != ILE_OK) return st;
    if (g_theta) CK(cudaMemcpyAsync(g_theta, d_th, sizeof(double) * nth, cudaMemcpyDeviceToHost, ctx->stream));
    if (gQ) CK(cudaMemcpyAsync(gQ, d_q, sizeof(double) * nq, cudaMemcpyDeviceToHost, ctx->stream));
    if (gU) CK(cudaMemcpyAsync(gU, d_u, sizeof(double) * nuv, cudaMemcpyDeviceToHost, ctx->stream));
    if (gV) CK(cudaMemcpyAsync(gV, d_v, sizeof(double) * nuv, cudaMemcpyDeviceToHost, ctx->stream));
    if (lnl) CK(cudaMemcpyAsync(lnl, d_l, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
    return finish_host_copies(ctx);
}

}  // namespace

extern "C" {

const char *ile_status_string(ile_status st) {
    switch (st) {
        case ILE_OK: return "ok";
        case ILE_E_ARG: return "invalid argument";
        case ILE_E_STATE: return "call out of order";
        case ILE_E_RANGE: return "interpolation index outside the extended time range";
        case ILE_E_NONFINITE: return "non-finite input or result";
        case ILE_E_CUDA: return "CUDA error";
        case ILE_E_NOMEM: return "device allocation failed";
        case ILE_E_TIMEOUT: return "device-side wait timed out";
    }
    return "unknown status";
}

const char *ile_last_error(const ile_ctx *ctx) { return ctx ? ctx->err : "null context"; }

ile_status ile_create(ile_ctx **out, int device, void *cuda_stream, ile_prec prec) {
    if (!out) return ILE_E_ARG;
    *out = nullptr;
    if (prec < ILE_PREC_FP32 || prec > ILE_PREC_BF16X3) return ILE_E_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return ILE_E_ARG;
    ile_ctx *ctx = new ile_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->prec = prec;
    DeviceGuard g(device);
    // flags[0]: the kernels' status bits; flags[1]: the check of the last ile_set_data's Q
    cudaError_t e = cudaMalloc((void **)&ctx->flags, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ctx->flags, 0, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->result, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        ile_status st = cuda_fail(ctx, e, "ile_create");
        ile_destroy(ctx);
        return st;
    }
    *out = ctx;
    return ILE_OK;
}

ile_status ile_destroy(ile_ctx *ctx) {
    if (!ctx) return ILE_OK;
    DeviceGuard g(ctx->device);
    void *bufs[] = {ctx->Qp,        ctx->UV,         ctx->Qquad,     ctx->dm_table,         ctx->Qtc[1][0], ctx->Qtc[1][1], ctx->Qtc[2][0],
                    ctx->Qtc[2][1],    ctx->s.C,        ctx->s.I0,      ctx->s.W,       ctx->s.A,
                    ctx->theta,        ctx->out,        ctx->lnp,       ctx->lnps,      ctx->part,
                    ctx->result,       ctx->flags,      ctx->keys,      ctx->buckets,   ctx->perm,
                    ctx->a_cdf,        ctx->a_lnps,     ctx->a_hist,    ctx->a_hist_fx, ctx->a_pooled,
                    ctx->a_iter_log,   ctx->a_iter_res, ctx->a_lnwp,    ctx->a_lnl,     ctx->a_iter,
                    ctx->a_bins,       ctx->pig,        ctx->gq_part,   ctx->guv_part,  ctx->g_in,
                    ctx->g_out,        ctx->g_cur,      ctx->g_bat,     ctx->g_tab,     ctx->g_part,
                    ctx->a_u,          ctx->Qadj[0],    ctx->Qadj[1],   ctx->Q64,       ctx->U64,
                    ctx->V64,          ctx->loud,       ctx->g2_cur,    ctx->g2_bat,    ctx->g2_tab,
                    ctx->g2_part,      ctx->a_upair,    ctx->ss_work};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (auto &v : ctx->ev)
        for (cudaEvent_t e : v) cudaEventDestroy(e);
    delete ctx;
    return ILE_OK;
}

ile_status ile_set_memory_limit(ile_ctx *ctx, size_t bytes) {
    if (!ctx) return ILE_E_ARG;
    ctx->mem_limit = bytes;
    return ILE_OK;
}

ile_status ile_memory_used(const ile_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return ILE_E_ARG;
    *bytes = ctx->mem_used;
    return ILE_OK;
}

ile_status ile_check_wait_timeout(ile_ctx *ctx, double timeout_s) {
    if (!ctx || !(timeout_s > 0.0) || !(timeout_s <= 10.0)) return ILE_E_ARG;
    DeviceGuard g(ctx->device);
    CK(ile_launch_wait_check(ctx->flags, timeout_s, ctx->stream));
    return read_flags(ctx);
}

ile_status ile_set_stream(ile_ctx *ctx, void *cuda_stream) {
    if (!ctx) return ILE_E_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return ILE_OK;
}

ile_status ile_set_refine(ile_ctx *ctx, int enable) {
    if (!ctx) return ILE_E_ARG;
    ctx->refine = enable != 0;
    return ILE_OK;
}

ile_status ile_refine_count(ile_ctx *ctx, int64_t *n) {
    if (!ctx || !n) return ILE_E_ARG;
    *n = 0;
    if (!ctx->loud) return ILE_OK;
    DeviceGuard g(ctx->device);
    int c = 0;
    CK(cudaMemcpyAsync(&c, ctx->loud, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *n = c;
    return ILE_OK;
}

ile_status ile_set_precision(ile_ctx *ctx, ile_prec prec) {
    if (!ctx || prec < ILE_PREC_FP32 || prec > ILE_PREC_BF16X3) return ILE_E_ARG;
    ctx->prec = prec;
    return ILE_OK;
}

}  // extern "C"

bool ile_sky_frame(const double pole[3], float rot[9]) {
    const double n = sqrt(pole[0] * pole[0] + pole[1] * pole[1] + pole[2] * pole[2]);
    if (!(n > 0.0) || !isfinite(n)) return false;
    const double p[3] = {pole[0] / n, pole[1] / n, pole[2] / n};
    double e1[3] = {-p[1], p[0], 0.0};  // z x p
    double m = sqrt(e1[0] * e1[0] + e1[1] * e1[1]);
    if (m < 1e-6) {
        e1[0] = 1.0;
        e1[1] = e1[2] = 0.0;
    } else {
        e1[0] /= m;
        e1[1] /= m;
    }
    const double e2[3] = {p[1] * e1[2] - p[2] * e1[1], p[2] * e1[0] - p[0] * e1[2], p[0] * e1[1] - p[1] * e1[0]};
    for (int r = 0; r < 3; r++) {
        rot[3 * r + 0] = (float)e1[r];
        rot[3 * r + 1] = (float)e2[r];
        rot[3 * r + 2] = (float)p[r];
    }
    return true;
}

// Pooled accumulators (max ln w, S1, S2, n) and the iteration log -> the summary fields of an
// ile_adapt_result (cdf and hist are filled by the caller).
void ile_fill_result(const double pooled[4], const double *ilog, int n_iter, ile_adapt_result *out) {
    for (int d = 0; d < ILE_NDIM; d++) {
        out->gmm_components[d] = 0;
        out->gmm_n[d] = 0.0;
        for (int c = 0; c < ILE_GMM_MAX; c++) out->gmm_w[d][c] = out->gmm_mu[d][c] = out->gmm_sigma[d][c] = 0.0;
    }
    out->gmm_pair_components = 0;
    out->gmm_pair_n = 0.0;
    for (int c = 0; c < ILE_GMM_MAX; c++) {
        out->gmm_pair_w[c] = 0.0;
        for (int j = 0; j < 2; j++) out->gmm_pair_mu[c][j] = 0.0;
        for (int j = 0; j < 3; j++) out->gmm_pair_cov[c][j] = 0.0;
    }
    out->max_lnw = pooled[0];
    out->s1 = pooled[1];
    out->s2 = pooled[2];
    out->n_total = pooled[3];
    out->n_iter = n_iter;
    for (int i = 0; i < ILE_ADAPT_LOG; i++) {
        out->iter_ln_L[i] = ilog[2 * i];
        out->iter_n_eff[i] = ilog[2 * i + 1];
    }
    const double Nd = pooled[3];
    if (Nd > 0) {
        const double mean = pooled[1] / Nd;
        double var = (pooled[2] - Nd * mean * mean) / (Nd - 1.0);
        if (var < 0.0) var = 0.0;
        out->ln_L = pooled[0] + log(mean);
        out->sigma_ln = Nd > 1 ? sqrt(var / Nd) / mean : INFINITY;
        out->n_eff = pooled[1];
        out->ess = pooled[1] * pooled[1] / pooled[2];
    } else {
        out->ln_L = -INFINITY;
        out->sigma_ln = INFINITY;
        out->n_eff = out->ess = 0.0;
    }
}

// Validate one intrinsic point and build its device-side description: PointParams, the FP32
// split rows Qp [K][2M][T_ext] and the packed U/V pairs [K][P][4] (shared by ile_set_data and
// the batched run).
ile_status ile_prepare_point(int n_det, int n_modes, const int *lm, const double *det_tensor,
                             const double *det_pos_m, const double *Q, int T_ext, double t_start_s, double fs_hz,
                             const double *U, const double *V, int n_window, double gmst_rad, double d_ref_mpc,
                             PointParams &pp_out, std::vector<float> &qp, std::vector<float> &uv,
                             std::vector<float> &quad, bool host_q) {
    if (!lm || !det_tensor || !det_pos_m || !Q || !U || !V) return ILE_E_ARG;
    if (n_det < 1 || n_det > ILE_MAX_DET || n_modes < 1 || n_modes > ILE_MAX_MODES) return ILE_E_ARG;
    if (n_window < 1 || n_window > ILE_MAX_WINDOW || T_ext < 2 || T_ext > ILE_MAX_TEXT) return ILE_E_ARG;
    if (!(fs_hz > 0) || !(d_ref_mpc > 0)) return ILE_E_ARG;
    if (!isfinite(t_start_s) || !isfinite(fs_hz) || !isfinite(gmst_rad) || !isfinite(d_ref_mpc)) return ILE_E_NONFINITE;
    const int K = n_det, M = n_modes, T = T_ext, R = 2 * M, P = M * (M + 1) / 2;
    PointParams pp{};
    pp.K = K;
    pp.M = M;
    pp.T_ext = T;
    pp.Nt = n_window;
    pp.x_offset = (float)(-t_start_s * fs_hz - 0.5 * n_window);
    pp.fs = (float)fs_hz;
    pp.gmst = (float)gmst_rad;
    pp.d_ref = (float)d_ref_mpc;
    pp.log_nt = (float)log((double)n_window);
    for (int a = 0; a < M; a++) {
        int l = lm[2 * a], m = lm[2 * a + 1];
        if (l < 2 || l > 4 || m < -l || m > l) return ILE_E_ARG;
        for (int b = 0; b < a; b++)
            if (lm[2 * b] == l && lm[2 * b + 1] == m) return ILE_E_ARG;
        if (!wigner_terms(l, m, pp.mode[a])) return ILE_E_ARG;
    }
    // (with host_q false, Q is converted and checked on the device by the caller)
    if (!finite_array(det_tensor, 9 * (size_t)K) || !finite_array(det_pos_m, 3 * (size_t)K) ||
        (host_q && !finite_array(Q, 2 * (size_t)K * M * T)) || !finite_array(U, 2 * (size_t)K * M * M) ||
        !finite_array(V, 2 * (size_t)K * M * M))
        return ILE_E_NONFINITE;
    for (int k = 0; k < K; k++) {
        for (int i = 0; i < 9; i++) pp.det_tensor[k][i] = (float)det_tensor[9 * k + i];
        for (int i = 0; i < 3; i++) pp.det_pos_c[k][i] = (float)(det_pos_m[3 * k + i] / ILE_C_SI);
    }
    qp.assign(host_q ? (size_t)K * R * T : 0, 0.f);
    for (int k = 0; k < K && host_q; k++)
        for (int a = 0; a < M; a++)
            for (int t = 0; t < T; t++) {
                const double *q = Q + 2 * (((size_t)k * M + a) * T + t);
                qp[((size_t)k * R + a) * T + t] = (float)q[0];
                qp[((size_t)k * R + M + a) * T + t] = (float)q[1];
            }
    uv.assign((size_t)K * P * 4, 0.f);
    for (int k = 0; k < K; k++) {
        int p = 0;
        for (int a = 0; a < M; a++)
            for (int b = a; b < M; b++, p++) {
                double f = (a == b) ? 1.0 : 2.0;  // conj(y_a) U_ab y_b + conj(y_b) U_ba y_a = 2 Re(...)
                const double *u = U + 2 * (((size_t)k * M + a) * M + b);
                const double *v = V + 2 * (((size_t)k * M + a) * M + b);
                float *o = &uv[((size_t)k * P + p) * 4];
                o[0] = (float)(f * u[0]);
                o[1] = (float)(f * u[1]);
                o[2] = (float)(f * v[0]);
                o[3] = (float)(f * v[1]);
            }
    }
    // real form of U_k and V_k for the quadratic-term MMA: operand row r = 2a + {0: Re c_a, 1: Im c_a};
    // output column 32 (b % 4) + 4 (b / 4) + p holds, for mode b, p = 0: Re z_b, 1: Im z_b
    // (z = U c), 2: Re w_b, 3: Im w_b (w = V c), so that the 32-column block g has everything of
    // the modes b = g, g + 4, ... (the modes math thread g of a sample forms the harmonics of)
    const int KPq = (R + 15) & ~15;
    quad.assign((size_t)K * KPq * ILE_QCOLS, 0.f);
    for (int k = 0; k < K; k++)
        for (int a = 0; a < M; a++)
            for (int b = 0; b < M; b++) {
                const double *u = U + 2 * (((size_t)k * M + b) * M + a);  // U_ba
                const double *v = V + 2 * (((size_t)k * M + b) * M + a);  // V_ba
                float *re = &quad[((size_t)k * KPq + 2 * a) * ILE_QCOLS];
                float *im = &quad[((size_t)k * KPq + 2 * a + 1) * ILE_QCOLS];
                const int c0 = 32 * (b % 4) + 4 * (b / 4);
                re[c0] = (float)u[0];
                im[c0] = (float)-u[1];
                re[c0 + 1] = (float)u[1];
                im[c0 + 1] = (float)u[0];
                re[c0 + 2] = (float)v[0];
                im[c0 + 2] = (float)-v[1];
                re[c0 + 3] = (float)v[1];
                im[c0 + 3] = (float)v[0];
            }
    pp_out = pp;
    return ILE_OK;
}

extern "C" {

ile_status ile_set_data(ile_ctx *ctx, int n_det, int n_modes, const int *lm, const double *det_tensor,
                        const double *det_pos_m, const double *Q, int T_ext, double t_start_s, double fs_hz,
                        const double *U, const double *V, int n_window, double gmst_rad, double d_ref_mpc) {
    if (!ctx) return ILE_E_ARG;
    PointParams pp{};
    std::vector<float> qp, uv, quad;
    // Q is converted to its FP32 rows (and checked) on the device, from the FP64 copy the
    // refinement keeps anyway
    ile_status st = ile_prepare_point(n_det, n_modes, lm, det_tensor, det_pos_m, Q, T_ext, t_start_s, fs_hz, U, V,
                                      n_window, gmst_rad, d_ref_mpc, pp, qp, uv, quad, false);
    if (st != ILE_OK) return st;
    DeviceGuard g(ctx->device);
    // the previous point's arrays are overwritten (or released and grown) below: no data until
    // that completes
    ctx->has_data = false;
    ctx->Qtc_ready[1] = ctx->Qtc_ready[2] = ctx->Qadj_ready = false;
    const size_t nqp = (size_t)n_det * 2 * n_modes * T_ext;
    CK(reserve(ctx, &ctx->Qp, sizeof(float) * nqp));
    CK(reserve(ctx, &ctx->UV, sizeof(float) * uv.size()));
    CK(reserve(ctx, &ctx->Qquad, sizeof(float) * quad.size()));
    const size_t nq = (size_t)n_det * n_modes * T_ext, nuv = (size_t)n_det * n_modes * n_modes;
    CK(reserve(ctx, &ctx->Q64, sizeof(double2) * nq));
    CK(reserve(ctx, &ctx->U64, sizeof(double2) * nuv));
    CK(reserve(ctx, &ctx->V64, sizeof(double2) * nuv));
    CK(cudaMemcpyAsync(ctx->Q64, Q, sizeof(double2) * nq, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->U64, U, sizeof(double2) * nuv, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->V64, V, sizeof(double2) * nuv, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->UV, uv.data(), sizeof(float) * uv.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->Qquad, quad.data(), sizeof(float) * quad.size(), cudaMemcpyHostToDevice, ctx->stream));
    unsigned *qchk = ctx->flags + 1, qbad = 0;
    CK(cudaMemsetAsync(qchk, 0, sizeof(unsigned), ctx->stream));
    CK(ile_launch_q_convert(reinterpret_cast<const double2 *>(ctx->Q64), n_det, n_modes, T_ext, ctx->Qp, qchk,
                            ctx->stream));
    CK(cudaMemcpyAsync(&qbad, qchk, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (qbad) return ILE_E_NONFINITE;  // the context stays without data
    ctx->pp = pp;
    ile_refine_params(n_det, n_modes, lm, det_tensor, det_pos_m, T_ext, t_start_s, fs_hz, n_window, gmst_rad,
                      d_ref_mpc, ctx->r64);  // validated above
    ctx->has_data = true;
    ctx->Qtc_ready[1] = ctx->Qtc_ready[2] = ctx->Qadj_ready = false;
    ctx->cap = ctx->cap;  // scratch is sized for ILE_MAX_DET x ILE_MAX_MODES, so it stays valid
    return ILE_OK;
}

ile_status ile_set_distance_marginalization(ile_ctx *ctx, int enable, double d_min_mpc, double d_max_mpc) {
    if (!ctx) return ILE_E_ARG;
    if (!ctx->has_data) return ILE_E_STATE;
    if (!enable) {
        ctx->pp.dm.on = 0;
        return ILE_OK;
    }
    if (!(d_min_mpc > 0.0) || !(d_max_mpc > d_min_mpc) || !isfinite(d_max_mpc)) return ILE_E_ARG;
    DeviceGuard g(ctx->device);
    if (!ctx->dm_table) CK(ctx_malloc(ctx, &ctx->dm_table, ile_dmarg_buffer_bytes()));
    DmargParams dm{};
    CK(ile_build_dmarg(d_min_mpc, d_max_mpc, (double)ctx->pp.d_ref, ctx->dm_table, dm, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->pp.dm = dm;
    return ILE_OK;
}

ile_status ile_build_quv(ile_ctx *ctx, int n_det, int n_modes, int64_t L, const double *h, const double *psd,
                         const double *d, double df, double f_low, double t_start_s, double fs_hz, int T_ext,
                         double *Q, double *U, double *V, unsigned flags) {
    if (!ctx || !h || !psd || !d || !Q || !U || !V) return ILE_E_ARG;
    if (n_det < 1 || n_det > ILE_MAX_DET || n_modes < 1 || n_modes > ILE_MAX_MODES) return ILE_E_ARG;
    if (L < 2 || L > ((int64_t)1 << 24) || T_ext < 1 || T_ext > ILE_MAX_TEXT) return ILE_E_ARG;
    if (!(df > 0.0) || !(fs_hz > 0.0) || !isfinite(f_low) || !isfinite(t_start_s)) return ILE_E_ARG;
    const int K = n_det, M = n_modes;
    const size_t nh = 2 * (size_t)M * L, nd = 2 * (size_t)K * L, ns = (size_t)K * L, nz = 2 * (size_t)K * M * L;
    const size_t nq = 2 * (size_t)K * M * T_ext, nuv = 2 * (size_t)K * M * M;
    DeviceGuard g(ctx->device);
    double *buf = nullptr;
    const bool dev = (flags & ILE_DEVICE_PTRS) != 0;
    const size_t n_all = nz + (dev ? 0 : nh + nd + ns + nq + 2 * nuv);
    CK(ctx_malloc(ctx, (void **)&buf, sizeof(double) * n_all));
    double *z = buf, *dh = (double *)h, *dp = (double *)psd, *dd = (double *)d, *dQ = Q, *dU = U, *dV = V;
    cudaError_t e = cudaSuccess;
    if (!dev) {
        dh = z + nz;
        dd = dh + nh;
        dp = dd + nd;
        dQ = dp + ns;
        dU = dQ + nq;
        dV = dU + nuv;
        e = cudaMemcpyAsync(dh, h, sizeof(double) * nh, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dd, d, sizeof(double) * nd, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dp, psd, sizeof(double) * ns, cudaMemcpyHostToDevice, ctx->stream);
    }
    if (e == cudaSuccess)
        e = ile_launch_quv(K, M, L, dh, dp, dd, df, f_low, t_start_s, fs_hz, T_ext, z, dQ, dU, dV, ctx->stream);
    if (e == cudaSuccess && !dev) {
        e = cudaMemcpyAsync(Q, dQ, sizeof(double) * nq, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(U, dU, sizeof(double) * nuv, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(V, dV, sizeof(double) * nuv, cudaMemcpyDeviceToHost, ctx->stream);
    }
    // the scratch is released after the work that uses it (stream-ordered wait)
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx_free(ctx, buf);
    CK(e);
    return ILE_OK;
}

ile_status ile_dmarg_eval(ile_ctx *ctx, const double *a, const double *b, int64_t n, double *out, unsigned flags) {
    if (!ctx || n < 0) return ILE_E_ARG;
    if (!ctx->pp.dm.on) return ILE_E_STATE;
    if (n == 0) return ILE_OK;
    if (!a || !b || !out) return ILE_E_ARG;
    DeviceGuard g(ctx->device);
    if (flags & ILE_DEVICE_PTRS) {
        CK(ile_launch_dmarg_eval(ctx->pp.dm, a, b, n, out, ctx->stream));
        return ILE_OK;
    }
    double *d = nullptr;
    CK(ctx_malloc(ctx, (void **)&d, sizeof(double) * 3 * (size_t)n));
    cudaError_t e = cudaMemcpyAsync(d, a, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + n, b, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = ile_launch_dmarg_eval(ctx->pp.dm, d, d + n, n, d + 2 * n, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, d + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx_free(ctx, d);
    CK(e);
    return ILE_OK;
}

ile_status ile_eval(ile_ctx *ctx, const double *samples, int64_t N, double *out, unsigned flags) {
    if (!ctx) return ILE_E_ARG;
    if (!ctx->has_data) return ILE_E_STATE;
    if (N < 0) return ILE_E_ARG;
    if (N == 0) return ILE_OK;
    if (!samples || !out) return ILE_E_ARG;
    const int full = (flags & ILE_NO_TMARG) ? 1 : 0;
    if (full && N > 65536) return ILE_E_ARG;
    const size_t out_elems = full ? (size_t)N * ctx->pp.Nt : (size_t)N;
    DeviceGuard g(ctx->device);
    ile_status st = ensure_samples(ctx, N);
    if (st != ILE_OK) return st;
    const bool nearest = (flags & ILE_NEAREST) != 0;
    if (flags & ILE_DEVICE_PTRS) return run_eval(ctx, samples, N, out, full, nearest);
    st = ensure_out(ctx, sizeof(double) * out_elems);
    if (st != ILE_OK) return st;
    CK(cudaMemcpyAsync(ctx->theta, samples, sizeof(double) * ILE_NDIM * (size_t)N, cudaMemcpyHostToDevice,
                       ctx->stream));
    st = run_eval(ctx, ctx->theta, N, ctx->out, full, nearest);
    if (st != ILE_OK) return st;
    st = read_flags(ctx);
    if (st != ILE_OK) return st;
    CK(cudaMemcpyAsync(out, ctx->out, sizeof(double) * out_elems, cudaMemcpyDeviceToHost, ctx->stream));
    return finish_host_copies(ctx);
}

ile_status ile_integrate(ile_ctx *ctx, const double *samples, const double *ln_prior, const double *ln_ps,
                         int64_t N, double *result, double *lnL_t_out, unsigned flags) {
    if (!ctx) return ILE_E_ARG;
    if (!ctx->has_data) return ILE_E_STATE;
    if (N < 1 || !samples || !result) return ILE_E_ARG;
    DeviceGuard g(ctx->device);
    ile_status st = ensure_samples(ctx, N);
    if (st != ILE_OK) return st;
    const int np = ile_mc_partial_count(N);
    if (flags & ILE_DEVICE_PTRS) {
        double *lnl = lnL_t_out;
        if (!lnl) {
            st = ensure_out(ctx, sizeof(double) * (size_t)N);
            if (st != ILE_OK) return st;
            lnl = ctx->out;
        }
        st = run_eval(ctx, samples, N, lnl, 0, (flags & ILE_NEAREST) != 0);
        if (st != ILE_OK) return st;
        StageScope t(ctx, 3, 2);
        CK(ile_launch_mc(lnl, ln_prior, ln_ps, N, ctx->part, np, result, ctx->stream));
        return ILE_OK;
    }
    st = ensure_out(ctx, sizeof(double) * (size_t)N);
    if (st != ILE_OK) return st;
    CK(cudaMemcpyAsync(ctx->theta, samples, sizeof(double) * ILE_NDIM * (size_t)N, cudaMemcpyHostToDevice,
                       ctx->stream));
    if (ln_prior)
        CK(cudaMemcpyAsync(ctx->lnp, ln_prior, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream));
    if (ln_ps) CK(cudaMemcpyAsync(ctx->lnps, ln_ps, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream));
    st = run_eval(ctx, ctx->theta, N, ctx->out, 0, (flags & ILE_NEAREST) != 0);
    if (st != ILE_OK) return st;
    {
        StageScope t(ctx, 3, 2);
        CK(ile_launch_mc(ctx->out, ln_prior ? ctx->lnp : nullptr, ln_ps ? ctx->lnps : nullptr, N, ctx->part, np,
                         ctx->result, ctx->stream));
    }
    st = read_flags(ctx);
    if (st != ILE_OK) return st;
    CK(cudaMemcpyAsync(result, ctx->result, 7 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (lnL_t_out) CK(cudaMemcpyAsync(lnL_t_out, ctx->out, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
    return finish_host_copies(ctx);
}

ile_status ile_eval_grad(ile_ctx *ctx, const double *samples, int64_t N, const double *g_lnL, double *g_samples,
                         double *g_Q, double *g_U, double *g_V, double *lnL_t_out, unsigned flags) {
    if (!ctx) return ILE_E_ARG;
    if (!ctx->has_data) return ILE_E_STATE;
    if (N < 0) return ILE_E_ARG;
    if (N == 0) return ILE_OK;
    if (!samples || !g_lnL) return ILE_E_ARG;
    if (!g_samples && !g_Q && !g_U && !g_V && !lnL_t_out) return ILE_E_ARG;
    if (N > ILE_GRAD_MAX_SAMPLES) return ILE_E_ARG;
    if (ctx->pp.dm.on) return ILE_E_STATE;  // the adjoint differentiates the time-marginalised likelihood
    DeviceGuard g(ctx->device);
    ile_status st = ensure_samples(ctx, N);
    if (st != ILE_OK) return st;
    if (flags & ILE_DEVICE_PTRS) return run_grad(ctx, samples, g_lnL, N, g_samples, g_Q, g_U, g_V, lnL_t_out);
    return run_grad_host(ctx, samples, g_lnL, N, g_samples, g_Q, g_U, g_V, lnL_t_out);
}

ile_status ile_integrate_grad(ile_ctx *ctx, const double *samples, const double *ln_prior, const double *ln_ps,
                              int64_t N, const double *g_scale, double *result, double *g_samples, double *g_Q,
                              double *g_U, double *g_V, unsigned flags) {
    if (!ctx) return ILE_E_ARG;
    if (!ctx->has_data) return ILE_E_STATE;
    if (N < 1 || !samples || !result) return ILE_E_ARG;
    if (N > ILE_GRAD_MAX_SAMPLES) return ILE_E_ARG;
    if (ctx->pp.dm.on) return ILE_E_STATE;
    DeviceGuard g(ctx->device);
    ile_status st = ensure_samples(ctx, N);
    if (st != ILE_OK) return st;
    st = ensure_out(ctx, sizeof(double) * (size_t)N);
    if (st != ILE_OK) return st;
    const int np = ile_mc_partial_count(N);
    const double *ds = samples, *dlp = ln_prior, *dlps = ln_ps;
    if (!(flags & ILE_DEVICE_PTRS)) {
        CK(cudaMemcpyAsync(ctx->theta, samples, sizeof(double) * ILE_NDIM * (size_t)N, cudaMemcpyHostToDevice,
                           ctx->stream));
        if (ln_prior) CK(cudaMemcpyAsync(ctx->lnp, ln_prior, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream));
        if (ln_ps) CK(cudaMemcpyAsync(ctx->lnps, ln_ps, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream));
        ds = ctx->theta;
        dlp = ln_prior ? ctx->lnp : nullptr;
        dlps = ln_ps ? ctx->lnps : nullptr;
    }
    st = run_eval(ctx, ds, N, ctx->out, 0);
    if (st != ILE_OK) return st;
    double *dres = (flags & ILE_DEVICE_PTRS) ? result : ctx->result;
    {
        StageScope t(ctx, 3, 3);
        CK(ile_launch_mc(ctx->out, dlp, dlps, N, ctx->part, np, dres, ctx->stream));
        const bool dev = (flags & ILE_DEVICE_PTRS) != 0;
        CK(ile_launch_mc_weights(ctx->out, dlp, dlps, N, dres, dev ? g_scale : nullptr,
                                 (!dev && g_scale) ? *g_scale : 1.0, ctx->g_in, ctx->stream));
    }
    if (flags & ILE_DEVICE_PTRS) return run_grad(ctx, ds, ctx->g_in, N, g_samples, g_Q, g_U, g_V, nullptr);
    const PointParams &pp = ctx->pp;
    const size_t nth = (size_t)ILE_NDIM * N, nq = 2 * (size_t)pp.K * pp.M * pp.T_ext,
                 nuv = 2 * (size_t)pp.K * pp.M * pp.M;
    CK(ensure_bytes(ctx, &ctx->g_out, &ctx->g_out_bytes, sizeof(double) * (nth + nq + 2 * nuv)));
    double *d_th = ctx->g_out, *d_q = d_th + nth, *d_u = d_q + nq, *d_v = d_u + nuv;
    st = run_grad(ctx, ds, ctx->g_in, N, g_samples ? d_th : nullptr, g_Q ? d_q : nullptr, g_U ? d_u : nullptr,
                  g_V ? d_v : nullptr, nullptr);
    if (st != ILE_OK) return st;
    st = read_flags(ctx);
    if (st != ILE_OK) return st;
    CK(cudaMemcpyAsync(result, ctx->result, 7 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (g_samples) CK(cudaMemcpyAsync(g_samples, d_th, sizeof(double) * nth, cudaMemcpyDeviceToHost, ctx->stream));
    if (g_Q) CK(cudaMemcpyAsync(g_Q, d_q, sizeof(double) * nq, cudaMemcpyDeviceToHost, ctx->stream));
    if (g_U) CK(cudaMemcpyAsync(g_U, d_u, sizeof(double) * nuv, cudaMemcpyDeviceToHost, ctx->stream));
    if (g_V) CK(cudaMemcpyAsync(g_V, d_v, sizeof(double) * nuv, cudaMemcpyDeviceToHost, ctx->stream));
    return finish_host_copies(ctx);
}

static ile_status adapt_alloc(ile_ctx *ctx, int64_t N) {
    // each fixed-size buffer is allocated once (a failed call leaves the rest for the next one)
    if (!ctx->a_cdf) CK(ctx_malloc(ctx, (void **)&ctx->a_cdf, sizeof(uint64_t) * ILE_NDIM * (ILE_NBINS + 1)));
    if (!ctx->a_lnps) CK(ctx_malloc(ctx, (void **)&ctx->a_lnps, sizeof(float) * ILE_NDIM * ILE_NBINS));
    if (!ctx->a_hist) {
        CK(ctx_malloc(ctx, (void **)&ctx->a_hist, sizeof(double) * ILE_NDIM * ILE_NBINS));
        CK(cudaMemset(ctx->a_hist, 0, sizeof(double) * ILE_NDIM * ILE_NBINS));
    }
    if (!ctx->a_hist_fx) {
        CK(ctx_malloc(ctx, (void **)&ctx->a_hist_fx, sizeof(unsigned long long) * ILE_NDIM * ILE_NBINS));
        CK(cudaMemset(ctx->a_hist_fx, 0, sizeof(unsigned long long) * ILE_NDIM * ILE_NBINS));
    }
    if (!ctx->a_pooled) CK(ctx_malloc(ctx, (void **)&ctx->a_pooled, sizeof(double) * 4));
    if (!ctx->a_iter_log) {
        CK(ctx_malloc(ctx, (void **)&ctx->a_iter_log, sizeof(double) * 2 * ILE_ADAPT_LOG));
        CK(cudaMemset(ctx->a_iter_log, 0, sizeof(double) * 2 * ILE_ADAPT_LOG));
    }
    if (!ctx->a_iter_res) CK(ctx_malloc(ctx, (void **)&ctx->a_iter_res, sizeof(double) * 8));
    if (!ctx->a_iter) CK(ctx_malloc(ctx, (void **)&ctx->a_iter, sizeof(int)));
    if (!ctx->g_cur) CK(ctx_malloc(ctx, (void **)&ctx->g_cur, sizeof(IleGmm) * ILE_NDIM));
    if (!ctx->g_bat) CK(ctx_malloc(ctx, (void **)&ctx->g_bat, sizeof(IleGmm) * ILE_NDIM));
    if (!ctx->g_tab) CK(ctx_malloc(ctx, (void **)&ctx->g_tab, sizeof(IleGmmTab) * ILE_NDIM));
    if (!ctx->g_part) CK(ctx_malloc(ctx, (void **)&ctx->g_part, sizeof(double) * ile_gmm_part_doubles()));
    if (ctx->sp.gmm_pair) {
        if (!ctx->g2_cur) CK(ctx_malloc(ctx, (void **)&ctx->g2_cur, sizeof(IleGmm2)));
        if (!ctx->g2_bat) CK(ctx_malloc(ctx, (void **)&ctx->g2_bat, sizeof(IleGmm2)));
        if (!ctx->g2_tab) CK(ctx_malloc(ctx, (void **)&ctx->g2_tab, sizeof(IleGmm2Tab)));
        if (!ctx->g2_part) CK(ctx_malloc(ctx, (void **)&ctx->g2_part, sizeof(double) * ile_gmm2_part_doubles()));
        if (N > ctx->a_upair_cap) {
            ctx->a_upair_cap = 0;
            CK(grow(ctx, &ctx->a_upair, sizeof(float) * 2 * (size_t)N));
            ctx->a_upair_cap = N;
        }
    }
    if (N > ctx->a_cap) {
        ctx->a_cap = 0;
        CK(grow(ctx, &ctx->a_lnwp, sizeof(double) * (size_t)N));
        CK(grow(ctx, &ctx->a_lnl, sizeof(double) * (size_t)N));
        CK(grow(ctx, &ctx->a_bins, (size_t)ILE_NDIM * (size_t)N));
        ctx->a_cap = N;
    }
    const size_t ub = sizeof(float) * (size_t)__builtin_popcount(ctx->sp.gmm_mask) * (size_t)N;
    if (ub > ctx->a_u_bytes) {
        ctx->a_u_bytes = 0;
        CK(grow(ctx, &ctx->a_u, ub));
        ctx->a_u_bytes = ub;
    }
    ile_status st = ensure_samples(ctx, N);
    if (st != ILE_OK) return st;
    return ILE_OK;
}

// Host form of the initial mixture (ile.h): C equal components evenly spaced over [lo, hi].
static IleGmm gmm_initial(int C, double lo, double hi) {
    IleGmm g{};
    g.C = C;
    g.lo = lo;
    g.hi = hi;
    for (int c = 0; c < C; c++) {
        g.w[c] = 1.0 / C;
        g.mu[c] = lo + (c + 0.5) * (hi - lo) / C;
        g.sigma[c] = (hi - lo) / C;
    }
    g.n = 0.0;
    return g;
}

ile_status ile_adapt_init(ile_ctx *ctx, const ile_adapt_cfg *cfg, const ile_adapt_result *resume) {
    if (!ctx || !cfg) return ILE_E_ARG;
    if (!ctx->has_data) return ILE_E_STATE;
    if (cfg->n_per_iter < 1 || cfg->n_per_iter > ((int64_t)1 << 23)) return ILE_E_ARG;
    if (!(cfg->eps > 0.0 && cfg->eps <= 1.0)) return ILE_E_ARG;
    if (cfg->adapt_mask >> ILE_NDIM) return ILE_E_ARG;
    if (cfg->sky_frame != 0 && cfg->sky_frame != 1) return ILE_E_ARG;
    for (int d = 0; d < ILE_NDIM; d++)
        if (!(cfg->hi[d] > cfg->lo[d]) || !isfinite(cfg->lo[d]) || !isfinite(cfg->hi[d])) return ILE_E_ARG;
    if (!(cfg->lo[5] > 0.0) || cfg->lo[1] < -1.0 || cfg->hi[1] > 1.0 || cfg->lo[3] < -1.0 || cfg->hi[3] > 1.0)
        return ILE_E_ARG;
    IleGmm gm[ILE_NDIM] = {};
    if (cfg->gmm_mask) {
        if (cfg->gmm_mask & ~cfg->adapt_mask) return ILE_E_ARG;
        if (cfg->gmm_components < 1 || cfg->gmm_components > ILE_GMM_MAX) return ILE_E_ARG;
        if (cfg->gmm_em_iters < 1 || cfg->gmm_em_iters > 100) return ILE_E_ARG;
        for (int d = 0; d < ILE_NDIM; d++) {
            if (!(cfg->gmm_mask & (1u << d))) continue;
            gm[d] = gmm_initial(cfg->gmm_components, cfg->lo[d], cfg->hi[d]);
            if (!resume) continue;
            if (resume->gmm_components[d] != cfg->gmm_components || !(resume->gmm_n[d] >= 0.0)) return ILE_E_ARG;
            for (int c = 0; c < cfg->gmm_components; c++) {
                const double w = resume->gmm_w[d][c], mu = resume->gmm_mu[d][c], sg = resume->gmm_sigma[d][c];
                if (!(w > 0.0) || !(sg > 0.0) || !isfinite(w) || !isfinite(sg) || !(mu >= cfg->lo[d]) ||
                    !(mu <= cfg->hi[d]))
                    return ILE_E_ARG;
                gm[d].w[c] = w;
                gm[d].mu[c] = mu;
                gm[d].sigma[c] = sg;
            }
            gm[d].n = resume->gmm_n[d];
        }
    }
    IleGmm2 g2{};
    if (cfg->gmm_pair) {
        // the sky pair drawn together: both variables adaptive and not in the separable mixtures
        if (cfg->gmm_pair != 1 || (cfg->adapt_mask & 3u) != 3u || (cfg->gmm_mask & 3u)) return ILE_E_ARG;
        if (cfg->gmm_components < 1 || cfg->gmm_components > ILE_GMM_MAX) return ILE_E_ARG;
        if (cfg->gmm_em_iters < 1 || cfg->gmm_em_iters > 100) return ILE_E_ARG;
        const double plo[2] = {cfg->lo[0], cfg->lo[1]}, phi[2] = {cfg->hi[0], cfg->hi[1]};
        ile_gmm2_init(g2, cfg->gmm_components, plo, phi);
        if (resume) {
            if (resume->gmm_pair_components != cfg->gmm_components || !(resume->gmm_pair_n >= 0.0)) return ILE_E_ARG;
            for (int c = 0; c < cfg->gmm_components; c++) {
                const double w = resume->gmm_pair_w[c], *mu = resume->gmm_pair_mu[c], *cv = resume->gmm_pair_cov[c];
                const double det = cv[0] * cv[2] - cv[1] * cv[1];
                if (!(w > 0.0) || !isfinite(w) || !(cv[0] > 0.0) || !(cv[2] > 0.0) || !(det > 0.0) ||
                    !isfinite(det))
                    return ILE_E_ARG;
                for (int j = 0; j < 2; j++)
                    if (!(mu[j] >= plo[j]) || !(mu[j] <= phi[j])) return ILE_E_ARG;
                g2.w[c] = w;
                for (int j = 0; j < 2; j++) g2.mu[c][j] = mu[j];
                for (int j = 0; j < 3; j++) g2.cov[c][j] = cv[j];
            }
            g2.n = resume->gmm_pair_n;
        }
    } else if (cfg->gmm_pair != 0) {
        return ILE_E_ARG;
    }
    DeviceGuard g(ctx->device);
    ctx->sp.gmm_mask = cfg->gmm_mask;  // sizes the mixture buffers in adapt_alloc
    ctx->sp.gmm_pair = cfg->gmm_pair;
    ile_status st = adapt_alloc(ctx, cfg->n_per_iter);
    if (st != ILE_OK) return st;
    IleSamplerParams sp{};
    for (int d = 0; d < ILE_NDIM; d++) {
        sp.lo[d] = (float)cfg->lo[d];
        sp.hi[d] = (float)cfg->hi[d];
    }
    sp.adapt_mask = cfg->adapt_mask;
    sp.key0 = (uint32_t)cfg->seed;
    sp.key1 = (uint32_t)(cfg->seed >> 32);
    sp.point = cfg->point_id;
    sp.gmst = ctx->pp.gmst;
    sp.sky = cfg->sky_frame;
    if (sp.sky && !ile_sky_frame(cfg->sky_pole, sp.rot)) return ILE_E_ARG;
    sp.gmm_mask = cfg->gmm_mask;
    sp.gmm_pair = cfg->gmm_pair;
    ctx->sp = sp;
    ctx->eps = cfg->eps;
    ctx->adapt_N = cfg->n_per_iter;
    ctx->gmm_iters = (cfg->gmm_mask || cfg->gmm_pair) ? cfg->gmm_em_iters : 0;
    CK(ile_launch_sampler_reset(sp, ctx->a_cdf, ctx->a_lnps, ctx->a_pooled, ctx->a_iter, 0, ctx->stream));
    if (sp.gmm_mask) {
        CK(cudaMemcpyAsync(ctx->g_cur, gm, sizeof gm, cudaMemcpyHostToDevice, ctx->stream));
        CK(ile_launch_gmm_table(sp.gmm_mask, ctx->g_cur, ctx->g_tab, ctx->stream));
        // gm is a stack array: the copy must finish before it goes out of scope
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (sp.gmm_pair) {
        CK(cudaMemcpyAsync(ctx->g2_cur, &g2, sizeof g2, cudaMemcpyHostToDevice, ctx->stream));
        CK(ile_launch_gmm2_table(ctx->g2_cur, ctx->g2_tab, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));  // g2 is a stack object
    }
    if (resume) {
        if (resume->n_iter < 0) return ILE_E_ARG;
        for (int d = 0; d < ILE_NDIM; d++) {
            const uint64_t *c = resume->cdf[d];
            if (c[0] != 0 || c[ILE_NBINS] != ((uint64_t)1 << 32)) return ILE_E_ARG;
            for (int b = 0; b < ILE_NBINS; b++)
                if (c[b + 1] <= c[b]) return ILE_E_ARG;
        }
        const double pooled[4] = {resume->max_lnw, resume->s1, resume->s2, resume->n_total};
        CK(cudaMemcpyAsync(ctx->a_cdf, resume->cdf, sizeof(resume->cdf), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->a_pooled, pooled, sizeof pooled, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->a_iter, &resume->n_iter, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        double ilog[2 * ILE_ADAPT_LOG];
        for (int i = 0; i < ILE_ADAPT_LOG; i++) {
            ilog[2 * i] = resume->iter_ln_L[i];
            ilog[2 * i + 1] = resume->iter_n_eff[i];
        }
        CK(cudaMemcpyAsync(ctx->a_iter_log, ilog, sizeof ilog, cudaMemcpyHostToDevice, ctx->stream));
        CK(ile_launch_lnps(sp, ctx->a_cdf, ctx->a_lnps, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    ctx->adapt_ready = true;
    return ILE_OK;
}

ile_status ile_adapt_step(ile_ctx *ctx, int n_iter) {
    if (!ctx || n_iter < 0) return ILE_E_ARG;
    if (!ctx->adapt_ready || !ctx->has_data) return ILE_E_STATE;
    DeviceGuard g(ctx->device);
    const int64_t N = ctx->adapt_N;
    ile_status st = adapt_alloc(ctx, N);
    if (st != ILE_OK) return st;
    const int np = ile_mc_partial_count(N);
    for (int it = 0; it < n_iter; it++) {
        {
            StageScope t(ctx, 0);
            CK(ile_launch_sample(ctx->sp, ctx->a_cdf, ctx->a_lnps, ctx->g_tab, ctx->g2_tab, ctx->a_iter, N,
                                 ctx->theta, ctx->a_lnwp, ctx->a_bins, ctx->a_u, ctx->a_upair, ctx->flags,
                                 ctx->stream));
        }
        st = run_eval(ctx, ctx->theta, N, ctx->a_lnl, 0);
        if (st != ILE_OK) return st;
        {
            StageScope t(ctx, 3, 2);
            CK(ile_launch_mc(ctx->a_lnl, ctx->a_lnwp, nullptr, N, ctx->part, np, ctx->a_iter_res, ctx->stream));
        }
        {
            StageScope t(ctx, 4, 2);
            CK(ile_launch_adapt(ctx->a_lnl, ctx->a_lnwp, ctx->a_bins, N, ctx->a_iter_res, ctx->sp, ctx->eps,
                                ctx->a_hist_fx, ctx->a_hist, ctx->a_cdf, ctx->a_lnps, ctx->a_pooled, ctx->a_iter_log,
                                ctx->a_iter, 1, ctx->stream));
        }
        if (ctx->sp.gmm_mask) {
            StageScope t(ctx, 4, 2 * ctx->gmm_iters);
            CK(ile_launch_gmm_update(ctx->sp.gmm_mask, ctx->a_u, ctx->a_lnl, ctx->a_lnwp, ctx->a_iter_res, N,
                                     ctx->gmm_iters, ctx->g_cur, ctx->g_bat, ctx->g_tab, ctx->g_part, ctx->stream));
        }
        if (ctx->sp.gmm_pair) {
            StageScope t(ctx, 4, 2 * ctx->gmm_iters);
            CK(ile_launch_gmm2_update(ctx->a_upair, ctx->a_lnl, ctx->a_lnwp, ctx->a_iter_res, N, ctx->gmm_iters,
                                      ctx->g2_cur, ctx->g2_bat, ctx->g2_tab, ctx->g2_part, ctx->stream));
        }
    }
    return ILE_OK;
}

ile_status ile_adapt_get(ile_ctx *ctx, ile_adapt_result *out) {
    if (!ctx || !out) return ILE_E_ARG;
    if (!ctx->adapt_ready) return ILE_E_STATE;
    DeviceGuard g(ctx->device);
    double pooled[4], ilog[2 * ILE_ADAPT_LOG];
    int it = 0;
    CK(cudaMemcpyAsync(pooled, ctx->a_pooled, sizeof pooled, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ilog, ctx->a_iter_log, sizeof ilog, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&it, ctx->a_iter, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(out->cdf, ctx->a_cdf, sizeof(out->cdf), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(out->hist, ctx->a_hist, sizeof(out->hist), cudaMemcpyDeviceToHost, ctx->stream));
    IleGmm gm[ILE_NDIM] = {};
    if (ctx->sp.gmm_mask) CK(cudaMemcpyAsync(gm, ctx->g_cur, sizeof gm, cudaMemcpyDeviceToHost, ctx->stream));
    IleGmm2 g2{};
    if (ctx->sp.gmm_pair) CK(cudaMemcpyAsync(&g2, ctx->g2_cur, sizeof g2, cudaMemcpyDeviceToHost, ctx->stream));
    ile_status st = read_flags(ctx);
    ile_fill_result(pooled, ilog, it, out);
    if (ctx->sp.gmm_pair) {
        out->gmm_pair_components = g2.C;
        for (int c = 0; c < g2.C; c++) {
            out->gmm_pair_w[c] = g2.w[c];
            for (int j = 0; j < 2; j++) out->gmm_pair_mu[c][j] = g2.mu[c][j];
            for (int j = 0; j < 3; j++) out->gmm_pair_cov[c][j] = g2.cov[c][j];
        }
        out->gmm_pair_n = g2.n;
    }
    for (int d = 0; d < ILE_NDIM; d++) {
        if (!(ctx->sp.gmm_mask & (1u << d))) continue;
        out->gmm_components[d] = gm[d].C;
        for (int c = 0; c < gm[d].C; c++) {
            out->gmm_w[d][c] = gm[d].w[c];
            out->gmm_mu[d][c] = gm[d].mu[c];
            out->gmm_sigma[d][c] = gm[d].sigma[c];
        }
        out->gmm_n[d] = gm[d].n;
    }
    return st;
}

ile_status ile_adapt_run(ile_ctx *ctx, const ile_adapt_cfg *cfg, ile_adapt_result *out) {
    if (!cfg || !out || cfg->n_iter < 1) return ILE_E_ARG;
    ile_status st = ile_adapt_init(ctx, cfg, nullptr);
    if (st != ILE_OK) return st;
    st = ile_adapt_step(ctx, cfg->n_iter);
    if (st != ILE_OK) return st;
    return ile_adapt_get(ctx, out);
}

ile_status ile_adapt_last(ile_ctx *ctx, double *theta, double *lnw_prior, uint8_t *bins, double *lnL_t) {
    if (!ctx) return ILE_E_ARG;
    if (!ctx->adapt_ready) return ILE_E_STATE;
    DeviceGuard g(ctx->device);
    const size_t N = (size_t)ctx->adapt_N;
    if (theta) CK(cudaMemcpyAsync(theta, ctx->theta, sizeof(double) * ILE_NDIM * N, cudaMemcpyDeviceToHost, ctx->stream));
    if (lnw_prior) CK(cudaMemcpyAsync(lnw_prior, ctx->a_lnwp, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
    if (bins) CK(cudaMemcpyAsync(bins, ctx->a_bins, ILE_NDIM * N, cudaMemcpyDeviceToHost, ctx->stream));
    if (lnL_t) CK(cudaMemcpyAsync(lnL_t, ctx->a_lnl, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
    return read_flags(ctx);
}

ile_status ile_merge_partials(int n_shards, const double *max_lnw, const double *s1, const double *s2,
                              const double *n, const double *hist, double *result, double *hist_out) {
    if (n_shards < 1 || !max_lnw || !s1 || !s2 || !n || !result) return ILE_E_ARG;
    double m = -INFINITY, N = 0.0;
    for (int i = 0; i < n_shards; i++) {
        if (!(n[i] >= 0.0)) return ILE_E_ARG;
        if (n[i] > 0.0) {
            m = fmax(m, max_lnw[i]);
            N += n[i];
        }
    }
    if (!(N > 0.0) || !isfinite(m)) return ILE_E_ARG;
    double S1 = 0.0, S2 = 0.0;
    if (hist_out)
        for (int j = 0; j < ILE_NDIM * ILE_NBINS; j++) hist_out[j] = 0.0;
    for (int i = 0; i < n_shards; i++) {
        if (n[i] <= 0.0) continue;
        const double f = exp(max_lnw[i] - m);
        S1 += s1[i] * f;
        S2 += s2[i] * f * f;
        if (hist && hist_out)
            for (int j = 0; j < ILE_NDIM * ILE_NBINS; j++) hist_out[j] += hist[(size_t)i * ILE_NDIM * ILE_NBINS + j] * f;
    }
    const double mean = S1 / N;
    double var = (S2 - N * mean * mean) / (N - 1.0);
    if (var < 0.0) var = 0.0;
    result[0] = m + log(mean);
    result[1] = N > 1 ? sqrt(var / N) / mean : INFINITY;
    result[2] = S1;
    result[3] = S1 * S1 / S2;
    result[4] = m;
    result[5] = S1;
    result[6] = S2;
    return ILE_OK;
}

ile_status ile_profile(ile_ctx *ctx, int enable) {
    if (!ctx) return ILE_E_ARG;
    ctx->profiling = enable != 0;
    return ILE_OK;
}

ile_status ile_profile_read(ile_ctx *ctx, double *out_ms, int64_t *out_count, int n_stages) {
    if (!ctx || !out_ms || n_stages < 0 || n_stages > ILE_NSTAGE) return ILE_E_ARG;
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    for (int s = 0; s < ILE_NSTAGE; s++) {
        double ms = 0.0;
        for (size_t i = 0; i + 1 < ctx->ev_used[s]; i += 2) {
            float f = 0.f;
            CK(cudaEventElapsedTime(&f, ctx->ev[s][i], ctx->ev[s][i + 1]));
            ms += f;
        }
        if (s < n_stages) {
            out_ms[s] = ms;
            if (out_count) out_count[s] = ctx->kernels[s];
        }
        ctx->ev_used[s] = 0;
        ctx->kernels[s] = 0;
    }
    return ILE_OK;
}

ile_status ile_sync(ile_ctx *ctx) {
    if (!ctx) return ILE_E_ARG;
    DeviceGuard g(ctx->device);
    return read_flags(ctx);
}

}  // extern "C"
