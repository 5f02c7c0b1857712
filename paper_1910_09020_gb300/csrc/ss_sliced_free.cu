// ss_sliced_free.cu -- pairs whose read and reference differ in length over
// the bit-sliced layout (reads of m bases, references of m_ref, uniform
// per batch): the walk of ss_sliced.cuh over the reference's m_ref columns
// with Section 2.4's correction -- the leading and trailing cells where a
// diagonal reads no base of the read are free, not obstacles.  Up to
// kSlicedMaxSegments batches of one threshold per launch, their CTAs one
// after another in the grid.
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
    int32_t mq;      // read bases
    int32_t mr;      // reference bases (!= mq)
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
    k_sliced_free(const __grid_constant__ SlicedArgs a)
{
    int s = 0;  // the CTA's segment (uniform across the CTA)
    while (s + 1 < a.nseg && blockIdx.x >= a.seg[s + 1].cta0)
        ++s;
    const SlicedSeg &sg = a.seg[s];
    __shared__ __align__(16)
        uint32_t vtab[SlicedEdges<E>::kRowsFree * SlicedShape<E>::WW];
    sliced_fill_edges2<E>(vtab, sg.mq, sg.mr);
    __syncthreads();
    const int64_t g =
        (int64_t)(blockIdx.x - sg.cta0) * kSlicedThreads + threadIdx.x;
    if (g >= sg.G)
        return;
    const int64_t p0 = g * 32;
    const int np = (int)min((int64_t)32, sg.n - p0);
    const uint32_t pad = np >= 32 ? 0u : 0xffffffffu << np;
    SlicedCount<E> cnt;
    sliced_walk2<E, true>(SlicedSrc{sg.q, sg.r, sg.G, g}, sg.mq, sg.mr, pad,
                          cnt, vtab, a.one);
    sliced_store<E>(cnt, sg.acc, sg.obs, p0, np, sg.vec != 0);
}

template <int E>
cudaError_t sliced_one(const SlicedArgs &a, unsigned grid, cudaStream_t st)
{
    k_sliced_free<E><<<grid, kSlicedThreads, 0, st>>>(a);
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

cudaError_t launch_sliced_free_segments(const SlicedSegment *segs, int nseg,
                                        int32_t E, cudaStream_t st)
{
    if (nseg <= 0)
        return cudaSuccess;
    if (nseg > kSlicedMaxSegments || E < 0 || E > kSlicedMaxE)
        return cudaErrorInvalidValue;
    SlicedArgs a;
    a.nseg = nseg;
    a.one = 1u;
    int64_t blocks = 0;
    for (int i = 0; i < nseg; ++i) {
        const SlicedSegment &s = segs[i];
        if (s.n <= 0 || s.m < 0 || s.m_ref < 0 || s.m == s.m_ref)
            return cudaErrorInvalidValue;
        SlicedSeg &d = a.seg[i];
        d.q = reinterpret_cast<const uint4 *>(s.reads);
        d.r = reinterpret_cast<const uint4 *>(s.refs);
        d.n = s.n;
        d.G = (s.n + 31) / 32;
        d.acc = s.acc;
        d.obs = s.obs;
        d.mq = s.m;
        d.mr = s.m_ref;
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
