// ss_rw_e3.cu -- instantiations of K3a for E = 25..31 (split across
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

cudaError_t launch_rw_uniform_e3(int E, const RwUniformArgs &a, size_t smem,
                                 unsigned grid, cudaStream_t st)
{
    switch (E) {
    case 25: return launch_one<25>(a, smem, grid, st);
    case 26: return launch_one<26>(a, smem, grid, st);
    case 27: return launch_one<27>(a, smem, grid, st);
    case 28: return launch_one<28>(a, smem, grid, st);
    case 29: return launch_one<29>(a, smem, grid, st);
    case 30: return launch_one<30>(a, smem, grid, st);
    case 31: return launch_one<31>(a, smem, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ssk
