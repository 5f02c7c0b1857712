// ss_rw_e0.cu -- instantiations of K3a for E = 0..9 (split across
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

cudaError_t launch_rw_uniform_e0(int E, const RwUniformArgs &a, size_t smem,
                                 unsigned grid, cudaStream_t st)
{
    switch (E) {
    case 0: return launch_one<0>(a, smem, grid, st);
    case 1: return launch_one<1>(a, smem, grid, st);
    case 2: return launch_one<2>(a, smem, grid, st);
    case 3: return launch_one<3>(a, smem, grid, st);
    case 4: return launch_one<4>(a, smem, grid, st);
    case 5: return launch_one<5>(a, smem, grid, st);
    case 6: return launch_one<6>(a, smem, grid, st);
    case 7: return launch_one<7>(a, smem, grid, st);
    case 8: return launch_one<8>(a, smem, grid, st);
    case 9: return launch_one<9>(a, smem, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ssk
