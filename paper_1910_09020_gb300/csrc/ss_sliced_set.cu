// ss_sliced_set.cu -- several thresholds, each from 0 to kSlicedSetMaxE, in
// one pass over the bit-sliced layout (sliced_walk_set): a threshold sweep's
// small thresholds, whose walks cost less than streaming the pairs, read the
// pairs once between them.  One kernel per set of two or more thresholds
// (26 sets of 0..4).
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "ss_device.cuh"
#include "ss_internal.h"
#include "ss_sliced.cuh"

namespace ssk {

namespace {

struct SlicedSetArgs {
    const uint4 *q;  // reads: uint4 index (blk * G + g) * 2 + b
    const uint4 *r;  // refs, same layout
    int64_t n;
    int64_t G;       // groups, ceil(n / 32)
    int32_t m;
    uint32_t one;    // 1 (see sliced_column)
    uint8_t *acc[kSlicedSetMaxE + 1];   // results of the set's I-th
    int32_t *obs[kSlicedSetMaxE + 1];   // threshold, ascending
    int32_t vec;     // every acc and obs 16-byte aligned
};

template <int I>
__device__ __forceinline__ void store_set(const SlicedTracks<> &,
                                          const SlicedSetArgs &, int64_t, int)
{
}

template <int I, int E, int... R>
__device__ __forceinline__ void store_set(const SlicedTracks<E, R...> &t,
                                          const SlicedSetArgs &a, int64_t p0,
                                          int np)
{
    sliced_store<E>(t.head.cnt, a.acc[I], a.obs[I], p0, np, a.vec != 0);
    store_set<I + 1>(t.tail, a, p0, np);
}

template <int... Es>
constexpr int max_of()
{
    int m = 0;
    ((m = Es > m ? Es : m), ...);
    return m;
}

template <int... Es>
__global__ void __launch_bounds__(kSlicedThreads)
    k_sliced_set(const SlicedSetArgs a)
{
    constexpr int EMAX = max_of<Es...>();
    __shared__ __align__(16)
        uint32_t vtab[SlicedEdges<EMAX>::kRows * SlicedShape<EMAX>::WW];
    sliced_fill_edges<EMAX>(vtab, a.m);
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * kSlicedThreads + threadIdx.x;
    if (g >= a.G)
        return;
    const int64_t p0 = g * 32;
    const int np = (int)min((int64_t)32, a.n - p0);
    const uint32_t pad = np >= 32 ? 0u : 0xffffffffu << np;
    SlicedTracks<Es...> t;
    sliced_walk_set<EMAX>(SlicedSrc{a.q, a.r, a.G, g}, a.m, pad, t, vtab,
                          a.one);
    store_set<0>(t, a, p0, np);
}

template <int... Es>
cudaError_t launch_set(const SlicedSetArgs &a, unsigned grid, cudaStream_t st,
                       std::integer_sequence<int, Es...>)
{
    k_sliced_set<Es...><<<grid, kSlicedThreads, 0, st>>>(a);
    return cudaGetLastError();
}

constexpr int popcount5(unsigned x)
{
    return (int)(x & 1u) + (int)((x >> 1) & 1u) + (int)((x >> 2) & 1u) +
           (int)((x >> 3) & 1u) + (int)((x >> 4) & 1u);
}

template <unsigned MASK>
cudaError_t launch_mask(const SlicedSetArgs &a, unsigned grid,
                        cudaStream_t st)
{
    if constexpr (popcount5(MASK) >= 2)
        return launch_set(a, grid, st,
                          typename MaskThresholds<MASK, 0>::type{});
    else
        return cudaErrorInvalidValue;
}

template <unsigned... M>
cudaError_t mask_dispatch(unsigned mask, const SlicedSetArgs &a, unsigned grid,
                          cudaStream_t st,
                          std::integer_sequence<unsigned, M...>)
{
    cudaError_t r = cudaErrorInvalidValue;
    ((mask == M ? (r = launch_mask<M>(a, grid, st), 0) : 0), ...);
    return r;
}

}  // namespace

cudaError_t launch_sliced_set(const uint32_t *reads, const uint32_t *refs,
                              int64_t n, int32_t m, unsigned mask,
                              uint8_t *const *acc, int32_t *const *obs,
                              cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    if (m < 0 || mask >= (1u << (kSlicedSetMaxE + 1)) ||
        popcount5(mask) < 2)
        return cudaErrorInvalidValue;
    const int64_t G = (n + 31) / 32;
    const int64_t blocks = (G + kSlicedThreads - 1) / kSlicedThreads;
    if (blocks > 0x7fffffff)
        return cudaErrorInvalidValue;
    SlicedSetArgs a;
    a.q = reinterpret_cast<const uint4 *>(reads);
    a.r = reinterpret_cast<const uint4 *>(refs);
    a.n = n;
    a.G = G;
    a.m = m;
    a.one = 1u;
    uintptr_t align = 0;
    for (int i = 0; i < popcount5(mask); ++i) {
        a.acc[i] = acc[i];
        a.obs[i] = obs[i];
        align |= (uintptr_t)acc[i] | (uintptr_t)obs[i];
    }
    a.vec = (align & 15) == 0;
    return mask_dispatch(
        mask, a, (unsigned)blocks, st,
        std::make_integer_sequence<unsigned,
                                   1u << (kSlicedSetMaxE + 1)>{});
}

}  // namespace ssk
