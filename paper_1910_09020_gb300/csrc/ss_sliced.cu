// ss_sliced.cu -- the plain launch over the bit-sliced layout: one thread
// per group of 32 pairs, the column walk of ss_sliced.cuh over all of them
// at once, then each pair's accept flag and min(count, E+1) written at its
// own index.
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "ss_device.cuh"
#include "ss_internal.h"
#include "ss_sliced.cuh"

namespace ssk {

namespace {

constexpr int kSlicedThreads = 128;

struct SlicedArgs {
    const uint4 *q;  // reads: uint4 index (blk * G + g) * 2 + b
    const uint4 *r;  // refs, same layout
    int64_t n;
    int64_t G;       // groups, ceil(n / 32)
    int32_t m;
    uint32_t one;    // 1 (see sliced_block)
    uint8_t *acc;
    int32_t *obs;
    int32_t vec;     // acc and obs 16-byte aligned: whole groups stored
                     // with 16-byte stores
};

// One group's words in global memory.
struct SlicedSrc {
    const uint4 *q, *r;
    int64_t G, g;
    __device__ __forceinline__ void load(const uint4 *base, int blk,
                                         uint32_t (&lo)[4],
                                         uint32_t (&hi)[4]) const
    {
        const uint4 *p = base + ((int64_t)blk * G + g) * 2;
        const uint4 a = __ldg(p), b = __ldg(p + 1);
        lo[0] = a.x, lo[1] = a.y, lo[2] = a.z, lo[3] = a.w;
        hi[0] = b.x, hi[1] = b.y, hi[2] = b.z, hi[3] = b.w;
    }
    __device__ __forceinline__ void query(int blk, int nb, uint32_t (&lo)[4],
                                          uint32_t (&hi)[4]) const
    {
        if (blk < 0 || blk >= nb) {
#pragma unroll
            for (int x = 0; x < 4; ++x)
                lo[x] = hi[x] = 0u;
            return;
        }
        load(q, blk, lo, hi);
    }
    __device__ __forceinline__ void ref(int blk, uint32_t (&lo)[4],
                                        uint32_t (&hi)[4]) const
    {
        load(r, blk, lo, hi);
    }
    // both planes of a block are 32 contiguous bytes: one L1 line each
    __device__ __forceinline__ void prefetch(int qblk, int rblk, int nb) const
    {
        if (qblk >= 0 && qblk < nb)
            asm volatile("prefetch.global.L1 [%0];"
                         :
                         : "l"(q + ((int64_t)qblk * G + g) * 2));
        if (rblk < nb)
            asm volatile("prefetch.global.L1 [%0];"
                         :
                         : "l"(r + ((int64_t)rblk * G + g) * 2));
    }
};

// Bytes 0..3 of the result: 1 for the pairs 4q..4q+3 of `ok` that are set.
__device__ __forceinline__ uint32_t flag_bytes(uint32_t ok, int q)
{
    return (((ok >> (4 * q)) & 0xfu) * 0x00204081u) & 0x01010101u;
}

template <int E>
__global__ void __launch_bounds__(kSlicedThreads) k_sliced(const SlicedArgs a)
{
    // the validity words of the edge blocks, the same for every thread
    using Ed = SlicedEdges<E>;
    constexpr int WW = SlicedShape<E>::WW;
    __shared__ __align__(16) uint32_t vtab[Ed::kRows * WW];
    {
        const Ed ed(a.m);
        for (int i = threadIdx.x; i < ed.rows() * WW; i += kSlicedThreads)
            vtab[i] = Ed::valid(ed.block_of(i / WW), i % WW, a.m);
    }
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * kSlicedThreads + threadIdx.x;
    if (g >= a.G)
        return;
    const int64_t p0 = g * 32;
    const int np = (int)min((int64_t)32, a.n - p0);
    const uint32_t pad = np >= 32 ? 0u : 0xffffffffu << np;
    SlicedCount<E> cnt;
    sliced_walk<E>(SlicedSrc{a.q, a.r, a.G, g}, a.m, pad, cnt, vtab, a.one);
    uint32_t cb[SlicedShape<E>::NB];
    cnt.bits(cb);
    const uint32_t ok = ~cnt.done();  // count <= E (Section 2.4 step 5)
    if (np == 32 && a.vec) {
        uint4 *o = reinterpret_cast<uint4 *>(a.obs + p0);
#pragma unroll
        for (int v = 0; v < 8; ++v)
            o[v] = make_uint4((uint32_t)sliced_count<E>(cb, 4 * v),
                              (uint32_t)sliced_count<E>(cb, 4 * v + 1),
                              (uint32_t)sliced_count<E>(cb, 4 * v + 2),
                              (uint32_t)sliced_count<E>(cb, 4 * v + 3));
        uint4 *f = reinterpret_cast<uint4 *>(a.acc + p0);
        f[0] = make_uint4(flag_bytes(ok, 0), flag_bytes(ok, 1),
                          flag_bytes(ok, 2), flag_bytes(ok, 3));
        f[1] = make_uint4(flag_bytes(ok, 4), flag_bytes(ok, 5),
                          flag_bytes(ok, 6), flag_bytes(ok, 7));
    } else {
        for (int i = 0; i < np; ++i) {
            a.obs[p0 + i] = sliced_count<E>(cb, i);
            a.acc[p0 + i] = (uint8_t)((ok >> i) & 1u);
        }
    }
}

template <int E>
cudaError_t sliced_one(const SlicedArgs &a, unsigned grid, cudaStream_t st)
{
    k_sliced<E><<<grid, kSlicedThreads, 0, st>>>(a);
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

cudaError_t launch_sliced(const uint32_t *reads, const uint32_t *refs,
                          int64_t n, int32_t m, int32_t E, uint8_t *acc,
                          int32_t *obs, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    if (E < 0 || E > kSlicedMaxE || m < 0)
        return cudaErrorInvalidValue;
    const int64_t G = (n + 31) / 32;
    const int64_t blocks = (G + kSlicedThreads - 1) / kSlicedThreads;
    if (blocks > 0x7fffffff)
        return cudaErrorInvalidValue;
    SlicedArgs a;
    a.q = reinterpret_cast<const uint4 *>(reads);
    a.r = reinterpret_cast<const uint4 *>(refs);
    a.n = n;
    a.G = G;
    a.m = m;
    a.one = 1u;
    a.acc = acc;
    a.obs = obs;
    a.vec = ((((uintptr_t)acc) | ((uintptr_t)obs)) & 15) == 0;
    return sliced_dispatch(E, a, (unsigned)blocks, st,
                           std::make_integer_sequence<int, kSlicedMaxE + 1>{});
}

}  // namespace ssk
