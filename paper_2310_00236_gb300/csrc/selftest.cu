// selftest.cu -- exercises the bounded-wait path of the pipelined kernels:
// one warp waits on an mbarrier that nothing arrives at, with a short poll
// limit, so the wait expires, the error word is set and the kernel returns.
// Nothing faults or hangs; the host then reads the error word like after any
// step.
#include <cuda_runtime.h>

#include "fused_common.cuh"
#include "wave_kernels.h"

namespace wave {

__global__ void selftest_wait_kernel(int *err, uint32_t polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) wait_phase_limit(&bar, 0, err, polls);  // no arrival: runs out
    __syncwarp();
}

cudaError_t selftest_wait(int *err, uint32_t polls, cudaStream_t st) {
    selftest_wait_kernel<<<1, 32, 0, st>>>(err, polls);
    return cudaGetLastError();
}

}  // namespace wave
