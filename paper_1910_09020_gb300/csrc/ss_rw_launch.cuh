// ss_rw_launch.cuh -- host side of the plain row-wise launches, compiled in
// each of the ss_rw_e*.cu translation units for its range of E.
#pragma once
#include <utility>

#include "ss_internal.h"
#include "ss_rw.cuh"

namespace ssk {

// One plain launch: the persistent pipelined kernel (pipe) or the staged
// kernel for long reads.
struct RwLaunch {
    bool pipe;
    RwPipeArgs pa;
    RwUniformArgs sa;
    size_t smem;
    unsigned grid;
};

template <int E>
cudaError_t rw_launch_one(const RwLaunch &L, cudaStream_t st)
{
    if (L.pipe)
        k_rw_uniform<E><<<L.grid, kRwThreads, L.smem, st>>>(L.pa);
    else
        k_rw_staged<E><<<L.grid, kRwThreads, L.smem, st>>>(L.sa);
    return cudaGetLastError();
}

// The staged kernel's shared-memory opt-in (once per process, before any
// stream capture).
template <int E>
cudaError_t rw_init_one()
{
    return cudaFuncSetAttribute(k_rw_staged<E>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                96 * 1024);
}

template <int LO, int... I>
cudaError_t rw_launch_range(int E, const RwLaunch &L, cudaStream_t st,
                            std::integer_sequence<int, I...>)
{
    cudaError_t r = cudaErrorInvalidValue;
    ((E == LO + I ? (r = rw_launch_one<LO + I>(L, st), 0) : 0), ...);
    return r;
}

template <int LO, int... I>
cudaError_t rw_init_range(std::integer_sequence<int, I...>)
{
    cudaError_t r = cudaSuccess;
    ((r == cudaSuccess ? (r = rw_init_one<LO + I>(), 0) : 0), ...);
    return r;
}

}  // namespace ssk
