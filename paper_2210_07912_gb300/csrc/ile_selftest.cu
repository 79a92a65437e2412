// ile_selftest.cu -- check of the bounded device-side waits (ile_check_wait_timeout): one block
// waits on an mbarrier phase that nothing completes, with the bounded sleeping wait the pipelined
// kernels use (try_wait with a suspend-time hint, a bounded number of tries); the wait gives up and
// raises ILE_FLAG_TIMEOUT, as a stalled pipeline would.  No fault or trap is involved.
#include "ile_internal.cuh"
#include "ile_tcgen05.cuh"

using namespace ile_tc;

namespace {

constexpr uint32_t SLEEP_NS = 10000;  // suspend-time hint per try, as in the pipelined kernels

// Nothing arrives on `bar`, so the wait must give up after `tries` tries (each returns no later
// than its suspend-time hint).
__global__ void wait_check_kernel(unsigned *flags, int tries) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_sleep(&bar, 0u, flags, 0u, tries, SLEEP_NS)) atomicOr(flags, ILE_FLAG_TIMEOUT);
}

}  // namespace

cudaError_t ile_launch_wait_check(unsigned *flags, double timeout_s, cudaStream_t st) {
    const double t = timeout_s * 1e9 / SLEEP_NS;
    const int tries = t < 1.0 ? 1 : t > 1e6 ? 1000000 : (int)t;
    wait_check_kernel<<<1, 32, 0, st>>>(flags, tries);
    return cudaGetLastError();
}
