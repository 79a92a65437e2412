// ile_batch.cu -- host side of the batched adaptive run (include/ile.h, ile_batch_*): hundreds of
// intrinsic points, each with its own Q/U/V, mode count, detector set, window, sample budget and
// sampler, integrated together.  One iteration is a fixed sequence of launches over the whole
// batch, captured once into a CUDA graph and replayed:
//   batched sampler (S0) -> batched delay sort -> the fused tensor-core kernel (S1-S5) as ONE
//   persistent launch over all (point, 128-sample tile) work items, largest first ->
//   batched Monte Carlo reduction (S6) -> batched histogram refit (S6).
// With FP32 or TF32x3 contraction arithmetic the contraction step is instead a per-point
// sequence of the single-point kernels (the plain comparison path), inside the same graph.
// The work-item order (longest first, cost ~ K N_t + K M^2 / 2 per tile), the B-ring depth and the
// job window width of the fused kernel are the tunables; ile_batch_tune times the admissible
// combinations on the batch's own samples and keeps the fastest.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "ile_internal.cuh"

struct ile_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    ile_prec prec = ILE_PREC_BF16X3;
    int n_points = 0;
    int64_t n_total = 0;
    int n_sm = 0;
    std::vector<PointParams> pps;
    std::vector<int64_t> N, off;
    std::vector<double> eps;
    // point data
    float *Qp = nullptr, *UV = nullptr, *Qquad = nullptr;
    std::vector<size_t> qp_off, uv_off, tc_off, quad_off;
    uint8_t *Qtc_hi = nullptr, *Qtc_lo = nullptr;
    double2 *Q64 = nullptr, *UV64 = nullptr;  // FP64 copies for the refinement of loud samples
    RefinePoint *rpts = nullptr;              // [n_points] (ile_refine.cu)
    int *loud = nullptr;                      // [2 n_total + 1] loud samples of the last iteration
    Tc2Point *pts = nullptr;
    IleBatchPoint *bp = nullptr;
    std::vector<IleBatchPoint> bp_host;
    // work lists
    int2 *items = nullptr, *blk256 = nullptr, *hblk = nullptr, *mblk = nullptr;
    int *mfirst = nullptr;
    int64_t n_items = 0;
    int n_blk256 = 0, n_hblk = 0, n_mblk = 0;
    // sampler state
    uint64_t *cdf = nullptr;
    float *lnps = nullptr;
    unsigned long long *hist_fx = nullptr;
    double *hist = nullptr, *pooled = nullptr, *iter_log = nullptr, *iter_res = nullptr;
    int *iter = nullptr;
    // per-sample arrays
    double *theta = nullptr, *lnwp = nullptr, *lnl = nullptr, *mc_part = nullptr;
    uint8_t *bins = nullptr;
    int *keys = nullptr, *perm = nullptr, *buckets = nullptr;
    // per-point scratch of the FP32 / TF32x3 contraction path
    IleScratch s{};
    int64_t s_cap = 0;
    unsigned *flags = nullptr;
    // fused-kernel configuration
    int LK = 0, LM = 0, LKP = 0;
    int a_tmem = 0, NB = 2, nwcol = 120, grid = 0;  // fused-kernel configuration (A placement, B ring, window)
    // graph of one iteration
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    char err[256] = {0};
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

ile_status fail(ile_batch *b, cudaError_t e, const char *where) {
    if (b) snprintf(b->err, sizeof b->err, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ILE_E_NOMEM : ILE_E_CUDA;
}

#define BK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return fail(b, e_, #call);         \
    } while (0)

template <typename T>
void release(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void free_points(ile_batch *b) {
    release(b->Qp);
    release(b->UV);
    release(b->Qquad);
    release(b->Qtc_hi);
    release(b->Qtc_lo);
    release(b->Q64);
    release(b->UV64);
    release(b->rpts);
    release(b->loud);
    release(b->pts);
    release(b->bp);
    release(b->items);
    release(b->blk256);
    release(b->hblk);
    release(b->mblk);
    release(b->mfirst);
    release(b->cdf);
    release(b->lnps);
    release(b->hist_fx);
    release(b->hist);
    release(b->pooled);
    release(b->iter_log);
    release(b->iter_res);
    release(b->iter);
    release(b->theta);
    release(b->lnwp);
    release(b->lnl);
    release(b->mc_part);
    release(b->bins);
    release(b->keys);
    release(b->perm);
    release(b->buckets);
    release(b->s.C);
    release(b->s.I0);
    release(b->s.W);
    release(b->s.A);
    b->s_cap = 0;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->n_points = 0;
}

void invalidate_graph(ile_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &v, cudaStream_t st) {
    cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * (v.empty() ? 1 : v.size()));
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
}

bool desc_ok(const ile_point_desc &d) {
    if (d.n_samples < 1 || d.n_samples > ((int64_t)1 << 23)) return false;
    if (!(d.eps > 0.0 && d.eps <= 1.0) || (d.adapt_mask >> ILE_NDIM)) return false;
    for (int k = 0; k < ILE_NDIM; k++)
        if (!(d.hi[k] > d.lo[k]) || !isfinite(d.lo[k]) || !isfinite(d.hi[k])) return false;
    if (!(d.lo[5] > 0.0) || d.lo[1] < -1.0 || d.hi[1] > 1.0 || d.lo[3] < -1.0 || d.hi[3] > 1.0) return false;
    if (d.sky_frame != 0 && d.sky_frame != 1) return false;
    if (d.sky_frame) {
        float rot[9];
        if (!ile_sky_frame(d.sky_pole, rot)) return false;
    }
    return true;
}

// One adaptive iteration over the whole batch, queued on the batch stream.
ile_status enqueue_iteration(ile_batch *b) {
    BK(ile_launch_batch_sample(b->bp, b->blk256, b->n_blk256, b->cdf, b->lnps, b->iter, b->theta, b->lnwp, b->bins,
                               b->stream));
    BK(ile_launch_batch_sort(b->n_points, b->bp, b->blk256, b->n_blk256, b->theta, b->keys, b->buckets, b->perm,
                             b->stream));
    // loud samples of every point are refined in FP64 after the contraction, exactly as in a
    // single-point run (so that each point's result equals that run bit for bit)
    BK(cudaMemsetAsync(b->loud, 0, sizeof(int), b->stream));
    const float thr = ile_refine_threshold((int)b->prec);
    if (b->prec == ILE_PREC_BF16X3) {
        BK(ile_launch_tc2_batch(b->pts, b->items, b->n_items, b->LK, b->LM, b->LKP, b->a_tmem, b->NB, b->nwcol, b->grid,
                                b->flags, b->stream));
    } else {
        for (int p = 0; p < b->n_points; p++) {
            const PointParams &pp = b->pps[p];
            const double *smp = b->theta + ILE_NDIM * b->off[p];
            const int *prm = b->perm + b->off[p];
            double *out = b->lnl + b->off[p];
            const int kp = ile_tc_kpad((int)b->prec, pp.M);
            if (b->prec == ILE_PREC_TF32X3 && ile_tc3_fits(pp.K, kp)) {
                // the fused TF32x3 kernel, as in a single-point run of this point
                BK(ile_launch_tc3(pp, b->Qtc_hi + b->tc_off[p], b->Qtc_lo + b->tc_off[p], ile_tc_tpad(pp.T_ext), kp,
                                  smp, prm, b->N[p], out, 0, LoudList{b->loud, thr, p, b->n_total}, b->flags,
                                  b->stream));
                continue;
            }
            BK(ile_launch_prep(pp, b->UV + b->uv_off[p], smp, prm, b->N[p], b->s, b->flags, b->stream));
            if (b->prec == ILE_PREC_FP32)
                BK(ile_launch_plain(pp, b->Qp + b->qp_off[p], b->s, prm, b->N[p], out, 0, LoudList{b->loud, thr, p, b->n_total},
                                    b->flags, b->stream));
            else
                BK(ile_launch_tc(b->prec, pp, b->Qtc_hi + b->tc_off[p], b->Qtc_lo + b->tc_off[p], b->s, prm, b->N[p],
                                 out, 0, LoudList{b->loud, thr, p, b->n_total}, b->flags, b->stream));
        }
    }
    BK(ile_launch_batch_refine(b->rpts, b->n_total, b->loud, b->n_total, b->flags, b->n_sm, b->stream));
    BK(ile_launch_batch_mc(b->n_points, b->bp, b->mblk, b->n_mblk, b->mfirst, b->lnl, b->lnwp, b->mc_part,
                           b->iter_res, b->stream));
    BK(ile_launch_batch_adapt(b->n_points, b->bp, b->hblk, b->n_hblk, b->lnl, b->lnwp, b->bins, b->iter_res,
                              b->hist_fx, b->hist, b->cdf, b->lnps, b->pooled, b->iter_log, b->iter, b->stream));
    return ILE_OK;
}

ile_status ensure_graph(ile_batch *b) {
    if (b->exec) return ILE_OK;
    BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    ile_status st = enqueue_iteration(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (st != ILE_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(b, e, "cudaStreamEndCapture");
    b->graph = g;
    BK(cudaGraphInstantiate(&b->exec, g, 0));
    return ILE_OK;
}

ile_status read_flags(ile_batch *b) {
    unsigned f = 0;
    BK(cudaMemcpyAsync(&f, b->flags, sizeof f, cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    if (f) BK(cudaMemsetAsync(b->flags, 0, sizeof(unsigned), b->stream));
    if (f & ILE_FLAG_TIMEOUT) return ILE_E_TIMEOUT;
    if (f & ILE_FLAG_RANGE) return ILE_E_RANGE;
    if (f & ILE_FLAG_NONFINITE) return ILE_E_NONFINITE;
    return ILE_OK;
}

}  // namespace

extern "C" {

ile_status ile_batch_create(ile_batch **out, int device, void *cuda_stream, ile_prec prec) {
    if (!out) return ILE_E_ARG;
    *out = nullptr;
    if (prec < ILE_PREC_FP32 || prec > ILE_PREC_BF16X3) return ILE_E_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return ILE_E_ARG;
    ile_batch *b = new ile_batch();
    b->device = device;
    b->prec = prec;
    DeviceGuard g(device);
    cudaError_t e = cudaSuccess;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        // a graph cannot be captured on the legacy default stream
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->flags, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->flags, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->grid, cudaDevAttrMultiProcessorCount, device);
    b->n_sm = b->grid;
    if (e != cudaSuccess) {
        ile_status st = fail(b, e, "ile_batch_create");
        ile_batch_destroy(b);
        return st;
    }
    *out = b;
    return ILE_OK;
}

ile_status ile_batch_destroy(ile_batch *b) {
    if (!b) return ILE_OK;
    DeviceGuard g(b->device);
    free_points(b);
    release(b->flags);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return ILE_OK;
}

const char *ile_batch_last_error(const ile_batch *b) { return b ? b->err : "null batch"; }

ile_status ile_batch_set_points(ile_batch *b, int n_points, const ile_point_desc *pts) {
    if (!b || !pts || n_points < 1 || n_points > ILE_BATCH_MAX_POINTS) return ILE_E_ARG;
    std::vector<PointParams> pps(n_points);
    std::vector<std::vector<float>> qps(n_points), uvs(n_points), quads(n_points);
    for (int p = 0; p < n_points; p++) {
        const ile_point_desc &d = pts[p];
        if (!desc_ok(d)) return ILE_E_ARG;
        ile_status st = ile_prepare_point(d.n_det, d.n_modes, d.lm, d.det_tensor, d.det_pos_m, d.Q, d.T_ext,
                                          d.t_start_s, d.fs_hz, d.U, d.V, d.n_window, d.gmst_rad, d.d_ref_mpc, pps[p],
                                          qps[p], uvs[p], quads[p]);
        if (st != ILE_OK) return st;
    }
    DeviceGuard g(b->device);
    BK(cudaStreamSynchronize(b->stream));
    free_points(b);
    const int split = b->prec == ILE_PREC_FP32 ? ILE_PREC_BF16X3 : (int)b->prec;  // tiles kept for BF16x3/TF32x3
    b->pps = pps;
    b->N.resize(n_points);
    b->off.resize(n_points);
    b->eps.resize(n_points);
    b->qp_off.resize(n_points);
    b->uv_off.resize(n_points);
    b->tc_off.resize(n_points);
    b->quad_off.resize(n_points);
    size_t qp_tot = 0, uv_tot = 0, tc_tot = 0, quad_tot = 0;
    int64_t ntot = 0;
    b->LK = b->LM = b->LKP = 0;
    for (int p = 0; p < n_points; p++) {
        const PointParams &pp = pps[p];
        b->N[p] = pts[p].n_samples;
        b->off[p] = ntot;
        ntot += pts[p].n_samples;
        b->eps[p] = pts[p].eps;
        b->qp_off[p] = qp_tot;
        qp_tot += qps[p].size();
        b->uv_off[p] = uv_tot;
        uv_tot += (uvs[p].size() + 3) / 4 * 4;
        b->quad_off[p] = quad_tot;
        quad_tot += quads[p].size();
        b->tc_off[p] = tc_tot;
        tc_tot += (ile_tc_q_bytes(split, pp.K, pp.M, pp.T_ext) + 255) / 256 * 256;
        b->LK = std::max(b->LK, pp.K);
        b->LM = std::max(b->LM, pp.M);
        b->LKP = std::max(b->LKP, ile_tc_kpad(ILE_PREC_BF16X3, pp.M));
    }
    b->n_total = ntot;
    // point data
    {
        std::vector<float> qp(qp_tot), uv(uv_tot, 0.f), quad(quad_tot);
        for (int p = 0; p < n_points; p++) {
            std::copy(qps[p].begin(), qps[p].end(), qp.begin() + b->qp_off[p]);
            std::copy(uvs[p].begin(), uvs[p].end(), uv.begin() + b->uv_off[p]);
            std::copy(quads[p].begin(), quads[p].end(), quad.begin() + b->quad_off[p]);
        }
        BK(upload(&b->Qp, qp, b->stream));
        BK(upload(&b->UV, uv, b->stream));
        BK(upload(&b->Qquad, quad, b->stream));
        BK(cudaStreamSynchronize(b->stream));
    }
    BK(cudaMalloc((void **)&b->Qtc_hi, tc_tot));
    BK(cudaMalloc((void **)&b->Qtc_lo, tc_tot));
    for (int p = 0; p < n_points; p++)
        BK(ile_launch_tc_split(split, pps[p], b->Qp + b->qp_off[p], b->Qquad + b->quad_off[p],
                               b->Qtc_hi + b->tc_off[p], b->Qtc_lo + b->tc_off[p], b->stream));
    // FP64 copies of Q, U, V for the refinement of loud samples: Q64 [sum K M T_ext], UV64 = U then V
    // of each point [2 sum K M^2]
    std::vector<size_t> q64_off(n_points), uv64_off(n_points);
    size_t q64_tot = 0, uv64_tot = 0;
    for (int p = 0; p < n_points; p++) {
        q64_off[p] = q64_tot;
        q64_tot += (size_t)pts[p].n_det * pts[p].n_modes * pts[p].T_ext;
        uv64_off[p] = uv64_tot;
        uv64_tot += 2 * (size_t)pts[p].n_det * pts[p].n_modes * pts[p].n_modes;
    }
    BK(cudaMalloc((void **)&b->Q64, sizeof(double2) * q64_tot));
    BK(cudaMalloc((void **)&b->UV64, sizeof(double2) * uv64_tot));
    for (int p = 0; p < n_points; p++) {
        const size_t nq = (size_t)pts[p].n_det * pts[p].n_modes * pts[p].T_ext,
                     nuv = (size_t)pts[p].n_det * pts[p].n_modes * pts[p].n_modes;
        BK(cudaMemcpyAsync(b->Q64 + q64_off[p], pts[p].Q, sizeof(double2) * nq, cudaMemcpyHostToDevice, b->stream));
        BK(cudaMemcpyAsync(b->UV64 + uv64_off[p], pts[p].U, sizeof(double2) * nuv, cudaMemcpyHostToDevice, b->stream));
        BK(cudaMemcpyAsync(b->UV64 + uv64_off[p] + nuv, pts[p].V, sizeof(double2) * nuv, cudaMemcpyHostToDevice,
                           b->stream));
    }
    BK(cudaMalloc((void **)&b->loud, sizeof(int) * (2 * (size_t)ntot + 1)));
    // per-sample arrays
    BK(cudaMalloc((void **)&b->theta, sizeof(double) * ILE_NDIM * ntot));
    BK(cudaMalloc((void **)&b->lnwp, sizeof(double) * ntot));
    BK(cudaMalloc((void **)&b->lnl, sizeof(double) * ntot));
    BK(cudaMalloc((void **)&b->bins, (size_t)ILE_NDIM * ntot));
    BK(cudaMalloc((void **)&b->keys, sizeof(int) * ntot));
    BK(cudaMalloc((void **)&b->perm, sizeof(int) * ntot));
    BK(cudaMalloc((void **)&b->buckets, sizeof(int) * ile_sort_key_buckets() * n_points));
    // sampler state
    BK(cudaMalloc((void **)&b->cdf, sizeof(uint64_t) * n_points * ILE_NDIM * (ILE_NBINS + 1)));
    BK(cudaMalloc((void **)&b->lnps, sizeof(float) * n_points * ILE_NDIM * ILE_NBINS));
    BK(cudaMalloc((void **)&b->hist_fx, sizeof(unsigned long long) * n_points * ILE_NDIM * ILE_NBINS));
    BK(cudaMalloc((void **)&b->hist, sizeof(double) * n_points * ILE_NDIM * ILE_NBINS));
    BK(cudaMalloc((void **)&b->pooled, sizeof(double) * 4 * n_points));
    BK(cudaMalloc((void **)&b->iter_log, sizeof(double) * 2 * ILE_ADAPT_LOG * n_points));
    BK(cudaMalloc((void **)&b->iter_res, sizeof(double) * 8 * n_points));
    BK(cudaMalloc((void **)&b->iter, sizeof(int) * n_points));
    // descriptors and work lists
    std::vector<Tc2Point> tp(n_points);
    std::vector<RefinePoint> rp(n_points);
    const float thr = ile_refine_threshold((int)b->prec);
    std::vector<IleBatchPoint> bph(n_points);
    std::vector<int2> items, blk256, hblk, mblk;
    std::vector<int> mfirst(n_points + 1, 0);
    std::vector<float> cost;
    const int TILE = ile_tc2_tile(), HC = ile_hist_chunk(), MC = ile_mc_chunk();
    for (int p = 0; p < n_points; p++) {
        const PointParams &pp = pps[p];
        const ile_point_desc &d = pts[p];
        Tc2Point &t = tp[p];
        t.pp = pp;
        t.Qhi = b->Qtc_hi + b->tc_off[p];
        t.Qlo = b->Qtc_lo + b->tc_off[p];
        t.UV = b->UV + b->uv_off[p];
        t.samples = b->theta + ILE_NDIM * b->off[p];
        t.perm = b->perm + b->off[p];
        t.out = b->lnl + b->off[p];
        t.N = b->N[p];
        t.TP = ile_tc_tpad(pp.T_ext);
        t.KP = ile_tc_kpad(ILE_PREC_BF16X3, pp.M);
        t.loud = LoudList{b->loud, thr, p, b->n_total};
        RefinePoint &r = rp[p];
        ile_refine_params(d.n_det, d.n_modes, d.lm, d.det_tensor, d.det_pos_m, d.T_ext, d.t_start_s, d.fs_hz,
                          d.n_window, d.gmst_rad, d.d_ref_mpc, r.r);
        r.r.thr = thr;
        const size_t nuv = (size_t)d.n_det * d.n_modes * d.n_modes;
        r.Q64 = b->Q64 + q64_off[p];
        r.U64 = b->UV64 + uv64_off[p];
        r.V64 = b->UV64 + uv64_off[p] + nuv;
        r.Qp = b->Qp + b->qp_off[p];
        r.samples = b->theta + ILE_NDIM * b->off[p];
        r.N = b->N[p];
        r.out = b->lnl + b->off[p];
        IleBatchPoint &q = bph[p];
        for (int k = 0; k < ILE_NDIM; k++) {
            q.sp.lo[k] = (float)d.lo[k];
            q.sp.hi[k] = (float)d.hi[k];
        }
        q.sp.adapt_mask = d.adapt_mask;
        q.sp.key0 = (uint32_t)d.seed;
        q.sp.key1 = (uint32_t)(d.seed >> 32);
        q.sp.point = d.point_id;
        q.sp.gmst = pp.gmst;
        q.sp.sky = d.sky_frame;
        if (d.sky_frame) ile_sky_frame(d.sky_pole, q.sp.rot);
        q.eps = d.eps;
        q.N = b->N[p];
        q.off = b->off[p];
        q.gmst = pp.gmst;
        const float c = (float)pp.K * pp.Nt + 0.5f * pp.K * pp.M * pp.M;
        for (int64_t t0 = 0; t0 < b->N[p]; t0 += TILE) {
            items.push_back(make_int2(p, (int)(t0 / TILE)));
            cost.push_back(c);
        }
        for (int64_t s0 = 0; s0 < b->N[p]; s0 += 256) blk256.push_back(make_int2(p, (int)s0));
        for (int64_t s0 = 0; s0 < b->N[p]; s0 += HC) hblk.push_back(make_int2(p, (int)s0));
        mfirst[p] = (int)mblk.size();
        for (int64_t s0 = 0; s0 < b->N[p]; s0 += MC) mblk.push_back(make_int2(p, (int)s0));
    }
    mfirst[n_points] = (int)mblk.size();
    // longest work first (stable: a point's tiles stay in order)
    std::vector<int64_t> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t c) { return cost[a] > cost[c]; });
    std::vector<int2> sorted(items.size());
    for (size_t i = 0; i < order.size(); i++) sorted[i] = items[order[i]];
    BK(upload(&b->pts, tp, b->stream));
    BK(upload(&b->rpts, rp, b->stream));
    BK(upload(&b->bp, bph, b->stream));
    BK(upload(&b->items, sorted, b->stream));
    BK(upload(&b->blk256, blk256, b->stream));
    BK(upload(&b->hblk, hblk, b->stream));
    BK(upload(&b->mblk, mblk, b->stream));
    BK(upload(&b->mfirst, mfirst, b->stream));
    BK(cudaMalloc((void **)&b->mc_part, sizeof(double) * 3 * std::max<size_t>(1, mblk.size())));
    b->bp_host = bph;
    b->n_items = (int64_t)sorted.size();
    b->n_blk256 = (int)blk256.size();
    b->n_hblk = (int)hblk.size();
    b->n_mblk = (int)mblk.size();
    if (b->prec != ILE_PREC_BF16X3) {
        const int64_t cap = *std::max_element(b->N.begin(), b->N.end());
        BK(cudaMalloc((void **)&b->s.C, sizeof(float) * (size_t)ILE_MAX_DET * 2 * ILE_MAX_MODES * cap));
        BK(cudaMalloc((void **)&b->s.I0, sizeof(int) * (size_t)ILE_MAX_DET * cap));
        BK(cudaMalloc((void **)&b->s.W, sizeof(float) * (size_t)ILE_MAX_DET * cap));
        BK(cudaMalloc((void **)&b->s.A, sizeof(float) * (size_t)cap));
        b->s_cap = cap;
    }
    // fused-kernel defaults: A operand in shared memory, deepest B ring that fits, the widest window
    int lo = 0, hi = 0;
    b->a_tmem = 0;
    b->nwcol = ile_tc2_nwcol_range(0, &lo, &hi);
    b->NB = 4;
    while (b->NB > 2 && !ile_tc2_batch_fits(0, b->LK, b->LM, b->LKP, b->NB)) b->NB--;
    BK(ile_launch_batch_reset(n_points, b->bp, b->cdf, b->lnps, b->pooled, b->iter, b->hist_fx, b->hist, b->iter_log,
                              b->stream));
    BK(cudaStreamSynchronize(b->stream));
    b->n_points = n_points;
    return ILE_OK;
}

ile_status ile_batch_reset(ile_batch *b) {
    if (!b) return ILE_E_ARG;
    if (!b->n_points) return ILE_E_STATE;
    DeviceGuard g(b->device);
    BK(ile_launch_batch_reset(b->n_points, b->bp, b->cdf, b->lnps, b->pooled, b->iter, b->hist_fx, b->hist,
                              b->iter_log, b->stream));
    return ILE_OK;
}

ile_status ile_batch_step(ile_batch *b, int n_iter) {
    if (!b || n_iter < 0) return ILE_E_ARG;
    if (!b->n_points) return ILE_E_STATE;
    DeviceGuard g(b->device);
    ile_status st = ensure_graph(b);
    if (st != ILE_OK) return st;
    for (int i = 0; i < n_iter; i++) BK(cudaGraphLaunch(b->exec, b->stream));
    return ILE_OK;
}

ile_status ile_batch_get(ile_batch *b, int first, int count, ile_adapt_result *out) {
    if (!b || !out || first < 0 || count < 0) return ILE_E_ARG;
    if (!b->n_points) return ILE_E_STATE;
    if (first + count > b->n_points) return ILE_E_ARG;
    if (count == 0) return ILE_OK;
    DeviceGuard g(b->device);
    const size_t nc = (size_t)ILE_NDIM * (ILE_NBINS + 1), nh = (size_t)ILE_NDIM * ILE_NBINS;
    std::vector<double> pooled(4 * (size_t)count), ilog(2 * ILE_ADAPT_LOG * (size_t)count);
    std::vector<int> it(count);
    std::vector<uint64_t> cdf(nc * count);
    std::vector<double> hist(nh * count);
    BK(cudaMemcpyAsync(pooled.data(), b->pooled + 4 * first, sizeof(double) * pooled.size(), cudaMemcpyDeviceToHost,
                       b->stream));
    BK(cudaMemcpyAsync(ilog.data(), b->iter_log + (size_t)2 * ILE_ADAPT_LOG * first, sizeof(double) * ilog.size(),
                       cudaMemcpyDeviceToHost, b->stream));
    BK(cudaMemcpyAsync(it.data(), b->iter + first, sizeof(int) * count, cudaMemcpyDeviceToHost, b->stream));
    BK(cudaMemcpyAsync(cdf.data(), b->cdf + nc * first, sizeof(uint64_t) * cdf.size(), cudaMemcpyDeviceToHost,
                       b->stream));
    BK(cudaMemcpyAsync(hist.data(), b->hist + nh * first, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost,
                       b->stream));
    ile_status st = read_flags(b);
    for (int i = 0; i < count; i++) {
        ile_adapt_result &r = out[i];
        ile_fill_result(&pooled[4 * (size_t)i], &ilog[2 * ILE_ADAPT_LOG * (size_t)i], it[i], &r);
        memcpy(r.cdf, &cdf[nc * i], sizeof(r.cdf));
        memcpy(r.hist, &hist[nh * i], sizeof(r.hist));
    }
    return st;
}

ile_status ile_batch_run(ile_batch *b, int n_points, const ile_point_desc *pts, int n_iter, ile_adapt_result *out) {
    if (!b || !out || n_iter < 1) return ILE_E_ARG;
    ile_status st = ile_batch_set_points(b, n_points, pts);
    if (st != ILE_OK) return st;
    st = ile_batch_step(b, n_iter);
    if (st != ILE_OK) return st;
    return ile_batch_get(b, 0, n_points, out);
}

ile_status ile_batch_last_samples(ile_batch *b, int point, double *theta, double *lnL_t) {
    if (!b || point < 0) return ILE_E_ARG;
    if (!b->n_points) return ILE_E_STATE;
    if (point >= b->n_points) return ILE_E_ARG;
    DeviceGuard g(b->device);
    const size_t N = (size_t)b->N[point], o = (size_t)b->off[point];
    if (theta)
        BK(cudaMemcpyAsync(theta, b->theta + ILE_NDIM * o, sizeof(double) * ILE_NDIM * N, cudaMemcpyDeviceToHost,
                           b->stream));
    if (lnL_t) BK(cudaMemcpyAsync(lnL_t, b->lnl + o, sizeof(double) * N, cudaMemcpyDeviceToHost, b->stream));
    return read_flags(b);
}

ile_status ile_batch_config(ile_batch *b, int a_tmem, int NB, int nwcol, int grid) {
    if (!b) return ILE_E_ARG;
    if (!b->n_points) return ILE_E_STATE;
    if (a_tmem != 0 && a_tmem != 1) return ILE_E_ARG;
    int lo = 0, hi = 0;
    ile_tc2_nwcol_range(a_tmem, &lo, &hi);
    if (NB < 2 || NB > 4 || nwcol < lo || nwcol > hi || grid < 1) return ILE_E_ARG;
    if (!ile_tc2_batch_fits(a_tmem, b->LK, b->LM, b->LKP, NB)) return ILE_E_ARG;
    b->a_tmem = a_tmem;
    b->NB = NB;
    b->nwcol = nwcol;
    b->grid = grid;
    invalidate_graph(b);
    return ILE_OK;
}

ile_status ile_batch_tune(ile_batch *b, int reps, ile_batch_tuning *out) {
    if (!b || reps < 1) return ILE_E_ARG;
    if (!b->n_points) return ILE_E_STATE;
    if (b->prec != ILE_PREC_BF16X3) return ILE_E_STATE;  // only the fused kernel has tunables
    DeviceGuard g(b->device);
    // samples to time on: one iteration (advances the samplers by one iteration)
    ile_status st = ile_batch_step(b, 1);
    if (st != ILE_OK) return st;
    int sms = 0;
    BK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    cudaEvent_t e0, e1;
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    float best = 1e30f;
    int bA = b->a_tmem, bNB = b->NB, bW = b->nwcol, n_tried = 0;
    auto time_one = [&](int A, int NB, int W, float &ms) -> cudaError_t {
        // a timed warm-up launch; a candidate already slower than twice the best is recorded at that
        // time, the others by `reps` more timed launches (each launch refills the loud-sample list:
        // its count is reset first)
        auto launch = [&]() {
            cudaError_t e = cudaMemsetAsync(b->loud, 0, sizeof(int), b->stream);
            if (e == cudaSuccess)
                e = ile_launch_tc2_batch(b->pts, b->items, b->n_items, b->LK, b->LM, b->LKP, A, NB, W, sms, b->flags,
                                         b->stream);
            return e;
        };
        ms = 0.f;
        cudaError_t e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) return e;
        if (ms <= 2.f * best) {
            e = cudaEventRecord(e0, b->stream);
            for (int r = 0; r < reps && e == cudaSuccess; r++) e = launch();
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) return e;
            ms /= reps;
        }
        if (out && n_tried < ILE_TUNE_MAX) {
            out->tried_a_tmem[n_tried] = A;
            out->tried_nb[n_tried] = NB;
            out->tried_nwcol[n_tried] = W;
            out->tried_ms[n_tried] = ms;
        }
        n_tried++;
        if (ms < best) {
            best = ms;
            bA = A;
            bNB = NB;
            bW = W;
        }
        return cudaSuccess;
    };
    // per A placement (shared memory, then TMEM when every point's operand fits): every window width
    // on an 8-column grid over the placement's admissible range (both ends included, widest first,
    // so that narrow windows, whose multi-window jobs cost several times more, are usually dismissed
    // after their warm-up launch) at the deepest B ring that fits, then the shallower rings at the
    // placement's best width
    cudaError_t e = cudaSuccess;
    for (int A = 0; A <= 1 && e == cudaSuccess; A++) {
        if (!ile_tc2_batch_fits(A, b->LK, b->LM, b->LKP, 2)) continue;
        int lo = 0, hi = 0;
        ile_tc2_nwcol_range(A, &lo, &hi);
        int nb_max = 2;
        for (int NB = 3; NB <= 4; NB++)
            if (ile_tc2_batch_fits(A, b->LK, b->LM, b->LKP, NB)) nb_max = NB;
        float abest = 1e30f;
        int aW = hi;
        for (int W = hi; e == cudaSuccess; W -= 8) {
            W = std::max(W, lo);
            float ms = 0.f;
            e = time_one(A, nb_max, W, ms);
            if (e == cudaSuccess && ms < abest) {
                abest = ms;
                aW = W;
            }
            if (W == lo) break;
        }
        for (int NB = 2; NB < nb_max && e == cudaSuccess; NB++) {
            float ms = 0.f;
            e = time_one(A, NB, aW, ms);
        }
    }
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(b, e, "ile_batch_tune");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st = read_flags(b);
    if (st != ILE_OK) return st;
    b->a_tmem = bA;
    b->NB = bNB;
    b->nwcol = bW;
    b->grid = sms;
    invalidate_graph(b);
    if (out) {
        out->a_tmem = bA;
        out->nb = bNB;
        out->nwcol = bW;
        out->grid = sms;
        out->ms = best;
        out->n_tried = std::min(n_tried, ILE_TUNE_MAX);
    }
    return ILE_OK;
}

}  // extern "C"
