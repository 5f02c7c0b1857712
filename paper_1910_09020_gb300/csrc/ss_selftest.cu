// ss_selftest.cu -- the context's status word, and the device-side bounded
// wait made to run out.
//
// k_status_take reads and clears the latched status word in one atomic
// exchange, so a flag that another stream's kernel latches at any moment is
// either taken by this read or left for the next one, never lost.
//
// One CTA initialises an mbarrier that nothing ever completes and waits on
// it with the same bounded wait the filter kernels use for their bulk
// copies.  The wait gives up after limit_ns and latches kStatusTimeout, which
// the host reads through ss_sync: the failure path of a wait, exercised
// without a fault, a trap or a hang.
#include <cuda_runtime.h>

#include <cstdint>

#include "ss_device.cuh"
#include "ss_internal.h"

namespace ssk {

__global__ void k_status_take(int *status, int *taken)
{
    *taken = atomicExch(status, 0);
}

cudaError_t launch_status_take(int *status, int *taken, cudaStream_t st)
{
    k_status_take<<<1, 1, 0, st>>>(status, taken);
    return cudaGetLastError();
}

__global__ void k_wait_timeout(uint64_t limit_ns, int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0)
        atomicOr(status, kStatusTimeout);
}

cudaError_t launch_wait_timeout(uint64_t limit_ns, int *status,
                                cudaStream_t st)
{
    k_wait_timeout<<<1, 32, 0, st>>>(limit_ns, status);
    return cudaGetLastError();
}

}  // namespace ssk
