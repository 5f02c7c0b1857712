// ss_rw_e2.cu -- instantiations of K3a for E = 18..24 (split across
// translation units so that they compile in parallel).
#include "ss_internal.h"
#include "ss_rw.cuh"

namespace ssk {

template <int E>
static cudaError_t launch_one(const RwUniformArgs &a, size_t smem,
                              unsigned grid, cudaStream_t st)
{
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(
            k_rw_uniform<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
            96 * 1024);
        if (e != cudaSuccess)
            return e;
        configured = true;
    }
    k_rw_uniform<E><<<grid, kRwThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rw_uniform_e2(int E, const RwUniformArgs &a, size_t smem,
                                 unsigned grid, cudaStream_t st)
{
    switch (E) {
    case 18: return launch_one<18>(a, smem, grid, st);
    case 19: return launch_one<19>(a, smem, grid, st);
    case 20: return launch_one<20>(a, smem, grid, st);
    case 21: return launch_one<21>(a, smem, grid, st);
    case 22: return launch_one<22>(a, smem, grid, st);
    case 23: return launch_one<23>(a, smem, grid, st);
    case 24: return launch_one<24>(a, smem, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ssk
