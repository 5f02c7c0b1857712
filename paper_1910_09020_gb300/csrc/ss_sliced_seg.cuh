// ss_sliced_seg.cuh -- the plain launch over the bit-sliced layout for up
// to kSlicedMaxSegments batches of one threshold (their CTAs one after
// another in one grid, each CTA finding its batch in the launch's table):
// k_sliced_seg<E, false> for reads and references of one length per batch
// (ss_sliced_multi.cu), k_sliced_seg<E, true> for references of another
// length than the reads, with Section 2.4's correction of the leading and
// trailing obstacles (ss_sliced_free.cu).  Kernels of their own, so that
// the single-batch launch keeps its registers.
#pragma once
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
    int32_t mr;      // reference bases
    int32_t vec;     // acc and obs 16-byte aligned
    uint32_t cta0;
};

struct SlicedSegArgs {
    SlicedSeg seg[kSlicedMaxSegments];
    int32_t nseg;
    uint32_t one;    // 1 (see sliced_column)
};

template <int E, bool FREE>
__global__ void __launch_bounds__(kSlicedThreads)
    k_sliced_seg(const __grid_constant__ SlicedSegArgs a)
{
    int s = 0;  // the CTA's batch (uniform across the CTA)
    while (s + 1 < a.nseg && blockIdx.x >= a.seg[s + 1].cta0)
        ++s;
    const SlicedSeg &sg = a.seg[s];
    constexpr int kRows =
        FREE ? SlicedEdges<E>::kRowsFree : SlicedEdges<E>::kRows;
    __shared__ __align__(16) uint32_t vtab[kRows * SlicedShape<E>::WW];
    if (FREE)
        sliced_fill_edges2<E>(vtab, sg.mq, sg.mr);
    else
        sliced_fill_edges<E>(vtab, sg.mq);
    __syncthreads();
    const int64_t g =
        (int64_t)(blockIdx.x - sg.cta0) * kSlicedThreads + threadIdx.x;
    if (g >= sg.G)
        return;
    const int64_t p0 = g * 32;
    const int np = (int)min((int64_t)32, sg.n - p0);
    const uint32_t pad = np >= 32 ? 0u : 0xffffffffu << np;
    SlicedCount<E> cnt;
    sliced_walk2<E, FREE>(SlicedSrc{sg.q, sg.r, sg.G, g}, sg.mq, sg.mr, pad,
                          cnt, vtab, a.one);
    sliced_store<E>(cnt, sg.acc, sg.obs, p0, np, sg.vec != 0);
}

template <bool FREE, int... I>
cudaError_t sliced_seg_dispatch(int E, const SlicedSegArgs &a, unsigned grid,
                                cudaStream_t st,
                                std::integer_sequence<int, I...>)
{
    cudaError_t r = cudaErrorInvalidValue;
    ((E == I ? (k_sliced_seg<I, FREE><<<grid, kSlicedThreads, 0, st>>>(a),
                r = cudaGetLastError(), 0)
             : 0),
     ...);
    return r;
}

// The launch over segs[0 .. nseg) (each n >= 1; m_ref the reference length,
// used with FREE; else the reads' m).
template <bool FREE>
cudaError_t sliced_seg_launch(const SlicedSegment *segs, int nseg, int32_t E,
                              cudaStream_t st)
{
    if (nseg <= 0)
        return cudaSuccess;
    if (nseg > kSlicedMaxSegments || E < 0 || E > kSlicedMaxE)
        return cudaErrorInvalidValue;
    SlicedSegArgs a;
    a.nseg = nseg;
    a.one = 1u;
    int64_t blocks = 0;
    for (int i = 0; i < nseg; ++i) {
        const SlicedSegment &s = segs[i];
        const int32_t mr = FREE ? s.m_ref : s.m;
        if (s.n <= 0 || s.m < 0 || mr < 0 || (FREE && s.m == mr))
            return cudaErrorInvalidValue;
        SlicedSeg &d = a.seg[i];
        d.q = reinterpret_cast<const uint4 *>(s.reads);
        d.r = reinterpret_cast<const uint4 *>(s.refs);
        d.n = s.n;
        d.G = (s.n + 31) / 32;
        d.acc = s.acc;
        d.obs = s.obs;
        d.mq = s.m;
        d.mr = mr;
        d.vec = ((((uintptr_t)s.acc) | ((uintptr_t)s.obs)) & 15) == 0;
        d.cta0 = (uint32_t)blocks;
        blocks += (d.G + kSlicedThreads - 1) / kSlicedThreads;
        if (blocks > 0x7fffffff)
            return cudaErrorInvalidValue;
    }
    return sliced_seg_dispatch<FREE>(
        E, a, (unsigned)blocks, st,
        std::make_integer_sequence<int, kSlicedMaxE + 1>{});
}

}  // namespace

}  // namespace ssk
