// ile_tc3.cu -- launcher of the fused TF32x3 tensor-core kernel (ile_tc2_kernel.cuh) for one
// intrinsic point.
//
// The BF16x3 kernel keeps its A operand (the tile's coefficients, hi and lo) in shared memory; in
// TF32 that operand doubles to 4 bytes per element and, with the B ring and the staging rows, no
// longer fits in 227 KB.  Here it lives in TMEM instead: 2 K KP of the 512 columns (288 for three
// detectors and 21 modes), each sample's row in its own lane, written by the sample's math threads
// with tcgen05.st and read by tcgen05.mma kind::tf32 as its A operand; the last 192 columns hold
// two 96-column accumulator buffers (windows of up to 89 columns).  Points whose A operand needs
// more than 320 columns (K KP > 160, e.g. four detectors with 21 modes) use the unfused kernel of
// ile_tc.cu.
#include "ile_tc2_kernel.cuh"

bool ile_tc3_fits(int K, int KP) {
    return K >= 1 && K <= ILE_MAX_DET && KP % 8 == 0 && acols_needed(OP_TF32_TMEM, K, KP) <= acol_of(OP_TF32_TMEM) &&
           tc2_smem<OP_TF32_TMEM>(K, 0, KP, 2, true) <= SMEM_LIMIT;  // (with the distance-marginalised store)
}

cudaError_t ile_launch_tc3(const PointParams &pp, const void *hi, const void *lo, int TP, int KP,
                           const double *samples, const int *perm, int64_t N, double *out, int full_grid,
                           LoudList loud, unsigned *flags, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    if (!ile_tc3_fits(pp.K, KP) || full_grid == 2) return cudaErrorInvalidConfiguration;
    const bool dm = pp.dm.on != 0;
    int NB = NBMAX;
    while (NB > 2 && tc2_smem<OP_TF32_TMEM>(pp.K, pp.M, KP, NB, dm) > SMEM_LIMIT) NB--;
    const size_t smem = tc2_smem<OP_TF32_TMEM>(pp.K, pp.M, KP, NB, dm);
    if (smem > SMEM_LIMIT) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(dm ? ile_tc2_kernel<false, true, OP_TF32_TMEM> : ile_tc2_kernel<false, false, OP_TF32_TMEM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // a window (plus up to 7 columns of 8-column alignment) must fit one accumulator buffer
    const int nwcol = bw_of(OP_TF32_TMEM) - 7;
    const int sms = sm_count();
    const int64_t ntiles = (N + TILE - 1) / TILE;
    const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
    Tc2Point one{};
    one.pp = pp;
    one.Qhi = hi;
    one.Qlo = lo;
    one.samples = samples;
    one.perm = perm;
    one.out = out;
    one.N = N;
    one.TP = TP;
    one.KP = KP;
    one.loud = (full_grid || pp.dm.on) ? LoudList{nullptr, 0.f, 0, 0} : loud;
    if (dm)
        ile_tc2_kernel<false, true, OP_TF32_TMEM><<<grid, NTHREADS, smem, st>>>(one, nullptr, nullptr, ntiles, pp.K, KP / 4,
                                                                        0, NB, nwcol, full_grid, flags);
    else
        ile_tc2_kernel<false, false, OP_TF32_TMEM><<<grid, NTHREADS, smem, st>>>(one, nullptr, nullptr, ntiles, pp.K, KP / 4,
                                                                         0, NB, nwcol, full_grid, flags);
    return cudaGetLastError();
}
