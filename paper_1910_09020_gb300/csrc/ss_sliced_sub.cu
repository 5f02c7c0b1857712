// ss_sliced_sub.cu -- the sub-maze mode (Section 2.5) over the bit-sliced
// layout: the walk of ss_sliced.cuh with every row restarting at each
// sub-maze's first column and at most y counted segments per sub-maze
// (SlicedSubMaze), 32 pairs per thread.
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "ss_device.cuh"
#include "ss_internal.h"
#include "ss_sliced.cuh"

namespace ssk {

namespace {

struct SlicedSubArgs {
    const uint4 *q;  // reads: uint4 index (blk * G + g) * 2 + b
    const uint4 *r;  // refs, same layout
    int64_t n;
    int64_t G;       // groups, ceil(n / 32)
    int32_t m;
    int32_t t;       // sub-maze width (columns)
    int32_t y;       // segments counted per sub-maze
    uint32_t one;    // 1 (see sliced_column)
    uint8_t *acc;
    int32_t *obs;
    int32_t vec;     // acc and obs 16-byte aligned
};

template <int E>
__global__ void __launch_bounds__(kSlicedThreads)
    k_sliced_sub(const SlicedSubArgs a)
{
    __shared__ __align__(16)
        uint32_t vtab[SlicedEdges<E>::kRows * SlicedShape<E>::WW];
    sliced_fill_edges<E>(vtab, a.m);
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * kSlicedThreads + threadIdx.x;
    if (g >= a.G)
        return;
    const int64_t p0 = g * 32;
    const int np = (int)min((int64_t)32, a.n - p0);
    const uint32_t pad = np >= 32 ? 0u : 0xffffffffu << np;
    SlicedCount<E> cnt;
    sliced_walk<E>(SlicedSrc{a.q, a.r, a.G, g}, a.m, pad, cnt, vtab, a.one,
                   SlicedSubMaze<E>(a.t, a.y));
    sliced_store<E>(cnt, a.acc, a.obs, p0, np, a.vec != 0);
}

template <int E>
cudaError_t sub_one(const SlicedSubArgs &a, unsigned grid, cudaStream_t st)
{
    k_sliced_sub<E><<<grid, kSlicedThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <int... I>
cudaError_t sub_dispatch(int E, const SlicedSubArgs &a, unsigned grid,
                         cudaStream_t st, std::integer_sequence<int, I...>)
{
    cudaError_t r = cudaErrorInvalidValue;
    ((E == I ? (r = sub_one<I>(a, grid, st), 0) : 0), ...);
    return r;
}

}  // namespace

cudaError_t launch_sliced_submaze(const uint32_t *reads, const uint32_t *refs,
                                  int64_t n, int32_t m, int32_t E, int32_t t,
                                  int32_t y, uint8_t *acc, int32_t *obs,
                                  cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    if (E < 0 || E > kSlicedMaxE || m < 0 || t < 1 || y < 1)
        return cudaErrorInvalidValue;
    const int64_t G = (n + 31) / 32;
    const int64_t blocks = (G + kSlicedThreads - 1) / kSlicedThreads;
    if (blocks > 0x7fffffff)
        return cudaErrorInvalidValue;
    SlicedSubArgs a;
    a.q = reinterpret_cast<const uint4 *>(reads);
    a.r = reinterpret_cast<const uint4 *>(refs);
    a.n = n;
    a.G = G;
    a.m = m;
    a.t = t;
    a.y = y;
    a.one = 1u;
    a.acc = acc;
    a.obs = obs;
    a.vec = ((((uintptr_t)acc) | ((uintptr_t)obs)) & 15) == 0;
    return sub_dispatch(E, a, (unsigned)blocks, st,
                        std::make_integer_sequence<int, kSlicedMaxE + 1>{});
}

}  // namespace ssk
