// Failure detection self-test (see lp_tv_selftest_wait in tvlp.h): one warp
// runs one of the kernels' bounded waits on a condition nothing satisfies,
// gives up after the kernels' limit, records the status the kernels record
// and returns, so a test can check the whole path (limit, status word, host
// read-back, a usable context afterwards) without faulting or hanging the GPU.
#include "tvlp.h"
#include "tvlp_kernels.cuh"

namespace tvlp {

__device__ unsigned g_tvlp_never_set = 0u;  // no kernel ever writes it

//   which 1: an mbarrier whose phase expects 16 bulk-copy bytes that are
//            never sent (no copy is issued, so nothing is in flight)
//   which 2: a progress counter that nothing increments
__global__ void __launch_bounds__(32) k_selftest_wait(int which, int *__restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    const int lane = threadIdx.x & 31;
    if (which == 1) {
        if (lane == 0) {
            mbar_init(&bar, 1);
            mbar_init_fence();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_expect_tx(&bar, 16u);
        __syncwarp();
        if (!mbar_wait_warp(&bar, 0u, kWaitLimit) && lane == 0) atomicExch(status, DEV_TIMEOUT_TMA);
    } else {
        (void)wait_counter(&g_tvlp_never_set, 1u, lane, status);
    }
}

}  // namespace tvlp

extern "C" int lp_tv_selftest_wait(int which, void *stream) {
    if (which != 1 && which != 2) return LP_EINVAL;
    int *status = tvlp::device_status_word();
    if (status == nullptr) return LP_ECUDA;
    tvlp::k_selftest_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(which, status);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ECUDA;
}
