// ile_tc2.cu -- launchers of the fused BF16x3 tensor-core kernel (ile_tc2_kernel.cuh) for one
// intrinsic point and for a batch of points in one persistent launch.
#include "ile_tc2_kernel.cuh"

namespace {

// One single-point launch of operand variant OP (DM: distance-marginalised epilogue; ADJ: the
// adjoint's D(n, j) pass with its per-sample outputs).
template <int OP, bool DM, bool ADJ = false>
cudaError_t launch_one(const PointParams &pp, const Tc2Point &one, int64_t ntiles, int KP, int full_grid,
                       unsigned *flags, cudaStream_t st) {
    int NB = NBMAX;
    while (NB > 2 && tc2_smem<OP>(pp.K, pp.M, KP, NB, DM) > SMEM_LIMIT) NB--;
    const size_t smem = tc2_smem<OP>(pp.K, pp.M, KP, NB, DM);
    if (smem > SMEM_LIMIT) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(ile_tc2_kernel<false, DM, OP, ADJ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // a window (plus up to 7 columns of 8-column alignment) fits one accumulator buffer
    const int nwcol = bw_of(OP) - 7 < NWCOL ? bw_of(OP) - 7 : NWCOL;
    const int sms = sm_count();
    const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
    ile_tc2_kernel<false, DM, OP, ADJ><<<grid, NTHREADS, smem, st>>>(one, nullptr, nullptr, ntiles, pp.K, KP / 8,
                                                                pp.M * (pp.M + 1) / 2, NB, nwcol, full_grid, flags);
    return cudaGetLastError();
}

}  // namespace

// The distance-marginalised launch takes the variant with its A operand in TMEM when the operand
// fits beside three accumulator buffers (K KP <= 176 columns: three detectors with all 21 modes);
// its epilogue exchanges values through shared memory between the threads of a sample, and keeping
// the tensor core's A reads off shared memory made that launch 10% faster (3.81 -> 3.41 ms per
// 2^20-sample iteration).  The plain launch keeps A in shared memory, which measured 2% faster
// there (1.633 against 1.670 ms per 2^20 samples).  Both give identical results.
cudaError_t ile_launch_tc2(const PointParams &pp, const void *hi, const void *lo, int TP, int KP, const float *UV,
                           const double *samples, const int *perm, int64_t N, double *out, float *grid_f,
                           int full_grid, LoudList loud, unsigned *flags, cudaStream_t st, const IleScratch *scr) {
    if (N <= 0) return cudaSuccess;
    const int64_t ntiles = (N + TILE - 1) / TILE;
    Tc2Point one{};
    one.pp = pp;
    one.Qhi = hi;
    one.Qlo = lo;
    one.UV = UV;
    one.samples = samples;
    one.perm = perm;
    one.out = out;
    one.grid_f = grid_f;
    if (full_grid == 2 && scr) {
        one.sC = scr->C;
        one.sI0 = scr->I0;
        one.sW = scr->W;
        one.sA = scr->A;
    }
    one.N = N;
    one.TP = TP;
    one.KP = KP;
    one.loud = (full_grid || pp.dm.on) ? LoudList{nullptr, 0.f, 0, 0} : loud;
    if (!pp.dm.on && full_grid == 2 && scr) return launch_one<OP_BF16_SMEM_N, false, true>(pp, one, ntiles, KP, 2, flags, st);
    if (!pp.dm.on) return launch_one<OP_BF16_SMEM_N, false>(pp, one, ntiles, KP, full_grid, flags, st);
    if (acols_needed(OP_BF16_TMEM, pp.K, KP) <= acol_of(OP_BF16_TMEM))
        return launch_one<OP_BF16_TMEM, true>(pp, one, ntiles, KP, full_grid, flags, st);
    return launch_one<OP_BF16_SMEM, true>(pp, one, ntiles, KP, full_grid, flags, st);
}

int ile_tc2_tile() { return TILE; }

// Batched launches: a_tmem 0 keeps the A operand in shared memory (three 128-column accumulator
// buffers), 1 puts it in TMEM (two 160-column buffers; needs K KP <= 192 for every point).
static int batch_op(int a_tmem) { return a_tmem ? OP_BF16_TMEM_W : OP_BF16_SMEM; }

size_t ile_tc2_batch_smem(int a_tmem, int LK, int LM, int LKP, int NB) {
    return a_tmem ? tc2_smem<OP_BF16_TMEM_W>(LK, LM, LKP, NB) : tc2_smem<OP_BF16_SMEM>(LK, LM, LKP, NB);
}

bool ile_tc2_batch_fits(int a_tmem, int LK, int LM, int LKP, int NB) {
    if (a_tmem && acols_needed(OP_BF16_TMEM_W, LK, LKP) > acol_of(OP_BF16_TMEM_W)) return false;
    return ile_tc2_batch_smem(a_tmem, LK, LM, LKP, NB) <= SMEM_LIMIT;
}

int ile_tc2_nwcol_range(int a_tmem, int *lo, int *hi) {
    *lo = NWCOL_MIN;
    *hi = bw_of(batch_op(a_tmem)) - 7;
    return *hi < NWCOL ? *hi : NWCOL;
}

cudaError_t ile_launch_tc2_batch(const Tc2Point *pts_dev, const int2 *items_dev, int64_t nitems, int LK, int LM,
                                 int LKP, int a_tmem, int NB, int nwcol, int grid, unsigned *flags, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    int lo = 0, hi = 0;
    ile_tc2_nwcol_range(a_tmem, &lo, &hi);
    if (NB < 2 || NB > NBMAX || nwcol < lo || nwcol > hi) return cudaErrorInvalidValue;
    if (!ile_tc2_batch_fits(a_tmem, LK, LM, LKP, NB)) return cudaErrorInvalidConfiguration;
    const size_t smem = ile_tc2_batch_smem(a_tmem, LK, LM, LKP, NB);
    auto kern = a_tmem ? ile_tc2_kernel<true, false, OP_BF16_TMEM_W> : ile_tc2_kernel<true, false, OP_BF16_SMEM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) grid = sm_count();
    if (grid > nitems) grid = (int)nitems;
    Tc2Point none{};
    kern<<<grid, NTHREADS, smem, st>>>(none, pts_dev, items_dev, nitems, LK, LKP / 8, LM * (LM + 1) / 2, NB, nwcol, 0,
                                        flags);
    return cudaGetLastError();
}
