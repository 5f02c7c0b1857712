// ss_rw_e1.cu -- instantiations of K3a for E = 10..17 (split across
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

cudaError_t launch_rw_uniform_e1(int E, const RwUniformArgs &a, size_t smem,
                                 unsigned grid, cudaStream_t st)
{
    switch (E) {
    case 10: return launch_one<10>(a, smem, grid, st);
    case 11: return launch_one<11>(a, smem, grid, st);
    case 12: return launch_one<12>(a, smem, grid, st);
    case 13: return launch_one<13>(a, smem, grid, st);
    case 14: return launch_one<14>(a, smem, grid, st);
    case 15: return launch_one<15>(a, smem, grid, st);
    case 16: return launch_one<16>(a, smem, grid, st);
    case 17: return launch_one<17>(a, smem, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ssk
