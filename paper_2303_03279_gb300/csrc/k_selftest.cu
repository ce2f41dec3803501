// k_selftest.cu - self-test of the bounded device wait (failure detection without a fault).
//
// One warp waits, through the same bounded-wait routine the streaming and tensor-core
// kernels use, on an mbarrier that nothing arrives at, with a short budget. The wait gives
// up, the kernel records the timeout in the session's control block and returns, exactly as
// a kernel whose bulk copy never landed would; the host then reads FC_ERR_TIMEOUT and the
// CUDA context stays usable. No copy is in flight and nothing faults.
#include "fc_internal.h"
#include "mbar.cuh"

namespace {

using namespace fcmbar;

__global__ void k_wait_probe(FcCtrl* ctrl, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);  // phase 0 never completes
    if (!ok && threadIdx.x == 0) atomicOr(&ctrl->timeout, 1);
}

}  // namespace

cudaError_t launch_wait_probe(FcCtrl* ctrl, unsigned long long limit_ns, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(ctrl, limit_ns);
    return cudaGetLastError();
}
