// ile_tc2.cu -- launchers of the fused BF16x3 tensor-core kernel (ile_tc2_kernel.cuh) for one
// intrinsic point and for a batch of points in one persistent launch.
#include "ile_tc2_kernel.cuh"

cudaError_t ile_launch_tc2(const PointParams &pp, const void *hi, const void *lo, int TP, int KP, const float *UV,
                           const double *samples, const int *perm, int64_t N, double *out, float *grid_f,
                           int full_grid, LoudList loud, unsigned *flags, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    int NB = NBMAX;
    while (NB > 2 && tc2_smem<false>(pp.K, pp.M, KP, NB) > SMEM_LIMIT) NB--;
    const size_t smem = tc2_smem<false>(pp.K, pp.M, KP, NB);
    if (smem > SMEM_LIMIT) return cudaErrorInvalidConfiguration;
    const bool dm = pp.dm.on != 0;
    cudaError_t e = cudaFuncSetAttribute(dm ? ile_tc2_kernel<false, true, false> : ile_tc2_kernel<false, false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    const int64_t ntiles = (N + TILE - 1) / TILE;
    const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
    Tc2Point one{};
    one.pp = pp;
    one.Qhi = hi;
    one.Qlo = lo;
    one.UV = UV;
    one.samples = samples;
    one.perm = perm;
    one.out = out;
    one.grid_f = grid_f;
    one.N = N;
    one.TP = TP;
    one.KP = KP;
    one.loud = (full_grid || pp.dm.on) ? LoudList{nullptr, 0.f, 0, 0} : loud;
    if (dm)
        ile_tc2_kernel<false, true, false><<<grid, NTHREADS, smem, st>>>(one, nullptr, nullptr, ntiles, pp.K, KP / 8,
                                                                  pp.M * (pp.M + 1) / 2, NB, NWCOL, full_grid, flags);
    else
        ile_tc2_kernel<false, false, false><<<grid, NTHREADS, smem, st>>>(one, nullptr, nullptr, ntiles, pp.K, KP / 8,
                                                                   pp.M * (pp.M + 1) / 2, NB, NWCOL, full_grid, flags);
    return cudaGetLastError();
}

int ile_tc2_tile() { return TILE; }

size_t ile_tc2_batch_smem(int LK, int LM, int LKP, int NB) { return tc2_smem<false>(LK, LM, LKP, NB); }

bool ile_tc2_batch_fits(int LK, int LM, int LKP, int NB) { return tc2_smem<false>(LK, LM, LKP, NB) <= SMEM_LIMIT; }

int ile_tc2_nwcol_range(int *lo, int *hi) {
    *lo = NWCOL_MIN;
    *hi = NWIN - 7;
    return NWCOL;
}

cudaError_t ile_launch_tc2_batch(const Tc2Point *pts_dev, const int2 *items_dev, int64_t nitems, int LK, int LM,
                                 int LKP, int NB, int nwcol, int grid, unsigned *flags, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    if (NB < 2 || NB > NBMAX || nwcol < NWCOL_MIN || nwcol > NWIN - 7) return cudaErrorInvalidValue;
    const size_t smem = tc2_smem<false>(LK, LM, LKP, NB);
    if (smem > SMEM_LIMIT) return cudaErrorInvalidConfiguration;
    cudaError_t e =
        cudaFuncSetAttribute(ile_tc2_kernel<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) grid = sm_count();
    if (grid > nitems) grid = (int)nitems;
    Tc2Point none{};
    ile_tc2_kernel<true, false, false><<<grid, NTHREADS, smem, st>>>(none, pts_dev, items_dev, nitems, LK, LKP / 8,
                                                       LM * (LM + 1) / 2, NB, nwcol, 0, flags);
    return cudaGetLastError();
}
