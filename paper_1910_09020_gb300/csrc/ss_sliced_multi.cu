// ss_sliced_multi.cu -- the plain launch of ss_sliced.cu over several
// batches of one threshold (their CTAs one after another in one grid): a
// batch mixing lengths, bucketed into uniform segments, in one launch per
// threshold.  A kernel of its own, so that the single-batch launch keeps
// its registers.
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "ss_device.cuh"
#include "ss_internal.h"
#include "ss_sliced.cuh"

namespace ssk {

namespace {

// One batch of a launch: its CTAs start at CTA cta0 of the grid.
struct SlicedSeg {
    const uint4 *q;  // reads: uint4 index (blk * G + g) * 2 + b
    const uint4 *r;  // refs, same layout
    int64_t n;
    int64_t G;       // groups, ceil(n / 32)
    uint8_t *acc;
    int32_t *obs;
    int32_t m;
    int32_t vec;     // acc and obs 16-byte aligned
    uint32_t cta0;
};

struct SlicedArgs {
    SlicedSeg seg[kSlicedMaxSegments];
    int32_t nseg;
    uint32_t one;    // 1 (see sliced_column)
};

template <int E>
__global__ void __launch_bounds__(kSlicedThreads)
    k_sliced_multi(const __grid_constant__ SlicedArgs a)
{
    int s = 0;  // the CTA's segment (uniform across the CTA)
    while (s + 1 < a.nseg && blockIdx.x >= a.seg[s + 1].cta0)
        ++s;
    const SlicedSeg &sg = a.seg[s];
    __shared__ __align__(16)
        uint32_t vtab[SlicedEdges<E>::kRows * SlicedShape<E>::WW];
    sliced_fill_edges<E>(vtab, sg.m);
    __syncthreads();
    const int64_t g =
        (int64_t)(blockIdx.x - sg.cta0) * kSlicedThreads + threadIdx.x;
    if (g >= sg.G)
        return;
    const int64_t p0 = g * 32;
    const int np = (int)min((int64_t)32, sg.n - p0);
    const uint32_t pad = np >= 32 ? 0u : 0xffffffffu << np;
    SlicedCount<E> cnt;
    sliced_walk<E>(SlicedSrc{sg.q, sg.r, sg.G, g}, sg.m, pad, cnt, vtab,
                   a.one);
    sliced_store<E>(cnt, sg.acc, sg.obs, p0, np, sg.vec != 0);
}

template <int E>
cudaError_t sliced_one(const SlicedArgs &a, unsigned grid, cudaStream_t st)
{
    k_sliced_multi<E><<<grid, kSlicedThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <int... I>
cudaError_t sliced_dispatch(int E, const SlicedArgs &a, unsigned grid,
                            cudaStream_t st, std::integer_sequence<int, I...>)
{
    cudaError_t r = cudaErrorInvalidValue;
    ((E == I ? (r = sliced_one<I>(a, grid, st), 0) : 0), ...);
    return r;
}

}  // namespace

cudaError_t launch_sliced_segments(const SlicedSegment *segs, int nseg,
                                   int32_t E, cudaStream_t st)
{
    if (nseg <= 0)
        return cudaSuccess;
    if (nseg > kSlicedMaxSegments || E < 0 || E > kSlicedMaxE)
        return cudaErrorInvalidValue;
    if (nseg == 1)
        return launch_sliced(segs[0].reads, segs[0].refs, segs[0].n,
                             segs[0].m, E, segs[0].acc, segs[0].obs, st);
    SlicedArgs a;
    a.nseg = nseg;
    a.one = 1u;
    int64_t blocks = 0;
    for (int i = 0; i < nseg; ++i) {
        const SlicedSegment &s = segs[i];
        if (s.n <= 0 || s.m < 0)
            return cudaErrorInvalidValue;
        SlicedSeg &d = a.seg[i];
        d.q = reinterpret_cast<const uint4 *>(s.reads);
        d.r = reinterpret_cast<const uint4 *>(s.refs);
        d.n = s.n;
        d.G = (s.n + 31) / 32;
        d.acc = s.acc;
        d.obs = s.obs;
        d.m = s.m;
        d.vec = ((((uintptr_t)s.acc) | ((uintptr_t)s.obs)) & 15) == 0;
        d.cta0 = (uint32_t)blocks;
        blocks += (d.G + kSlicedThreads - 1) / kSlicedThreads;
        if (blocks > 0x7fffffff)
            return cudaErrorInvalidValue;
    }
    return sliced_dispatch(E, a, (unsigned)blocks, st,
                           std::make_integer_sequence<int, kSlicedMaxE + 1>{});
}

}  // namespace ssk
