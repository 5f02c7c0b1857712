// ss_compact.cu -- downstream pass-through: the pairs the filter accepts
// ("sequence alignment is needed", Section 2.4 step 5) compacted, in order,
// into an index list an aligner can consume, and their packed sequences
// gathered into dense buffers.
//
// Three passes, no host synchronisation: per-CTA counts of accepted pairs,
// an exclusive scan of the CTA counts (one CTA), and a scatter in which each
// CTA writes its accepted indices at its offset.  A thread takes 16
// consecutive flags (one 16-byte load where the flags are aligned) as a
// 16-bit mask; ranks inside the CTA come from a scan of the threads' mask
// counts.
#include <cuda_runtime.h>

#include <cstdint>

#include "ss_device.cuh"
#include "ss_internal.h"

namespace ssk {

constexpr int kCompactThreads = 256;
constexpr int kCompactItems = 16;  // pairs per thread
constexpr int kCompactChunk = kCompactThreads * kCompactItems;

// Flags p0 .. p0+15 (those below n) as a mask: bit k set when flag p0 + k
// is nonzero.
__device__ __forceinline__ uint32_t compact_mask16(const uint8_t *acc,
                                                   int64_t n, int64_t p0)
{
    uint32_t mask = 0u;
    if (p0 + 16 <= n && ((uintptr_t)(acc + p0) & 15) == 0) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(acc + p0));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // bit 7 of each byte: the byte is nonzero
            const uint32_t nz =
                (((w[q] & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w[q]) & 0x80808080u;
            // bits 7, 15, 23, 31 -> bits 4q .. 4q+3
            const uint32_t b = (nz >> 7) & 0x01010101u;
            mask |= ((b * 0x01020408u) >> 24 & 0xfu) << (4 * q);
        }
    } else {
        for (int k = 0; k < 16; ++k)
            if (p0 + k < n && acc[p0 + k])
                mask |= 1u << k;
    }
    return mask;
}

__global__ void __launch_bounds__(kCompactThreads)
    k_compact_count(const uint8_t *__restrict__ acc, int64_t n,
                    int64_t *__restrict__ block_counts)
{
    __shared__ int warp_sums[kCompactThreads / 32];
    const int64_t p0 = (int64_t)blockIdx.x * kCompactChunk +
                       (int64_t)threadIdx.x * kCompactItems;
    int c = __popc(compact_mask16(acc, n, p0));
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0)
        warp_sums[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kCompactThreads / 32; ++w)
            t += warp_sums[w];
        block_counts[blockIdx.x] = t;
    }
}

// Exclusive scan of nb CTA counts in place; writes the total to *total.
__global__ void __launch_bounds__(1024)
    k_compact_scan(int64_t *__restrict__ block_counts, int64_t nb,
                   int64_t *__restrict__ total)
{
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t per = (nb + 1023) / 1024;
    const int64_t lo = t * per, hi = lo + per < nb ? lo + per : nb;
    int64_t s = 0;
    for (int64_t b = lo; b < hi; ++b)
        s += block_counts[b];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - s;
    for (int64_t b = lo; b < hi; ++b) {
        const int64_t c = block_counts[b];
        block_counts[b] = run;
        run += c;
    }
    if (t == 1023)
        *total = part[1023];
}

__global__ void __launch_bounds__(kCompactThreads)
    k_compact_scatter(const uint8_t *__restrict__ acc, int64_t n,
                      const int64_t *__restrict__ block_offsets,
                      int64_t *__restrict__ out_index)
{
    __shared__ int warp_sums[kCompactThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * kCompactChunk +
                       (int64_t)threadIdx.x * kCompactItems;
    uint32_t mask = compact_mask16(acc, n, p0);
    const int c = __popc(mask);
    // inclusive scan of the counts over the warp, then over the warps
    int x = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off)
            x += y;
    }
    if (lane == 31)
        warp_sums[warp] = x;
    __syncthreads();
    int before = 0;
#pragma unroll
    for (int w = 0; w < kCompactThreads / 32; ++w)
        before += w < warp ? warp_sums[w] : 0;
    int64_t o = block_offsets[blockIdx.x] + before + (x - c);
    // the thread's accepted indices, in order
    while (mask) {
        const int k = __ffs(mask) - 1;
        mask &= mask - 1u;
        out_index[o++] = p0 + k;
    }
}

// Dense copy of the selected fixed-stride pairs: slot i <- pair index[i],
// for i < min(*count, n); the outputs hold n slots and the sources n pairs.
// A warp copies 32 slots at a time: lane l holds slot i0 + l's source
// index, and the 32 * w16 words are spread over the lanes in output order,
// so every store instruction writes 32 consecutive words.
__global__ void k_gather_pairs(const uint32_t *__restrict__ reads,
                               const uint32_t *__restrict__ refs, int w16,
                               uint32_t w16_magic,
                               const int64_t *__restrict__ index,
                               const int64_t *__restrict__ count,
                               uint32_t *__restrict__ out_reads,
                               uint32_t *__restrict__ out_refs, int64_t n)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = *count;
    const int64_t cnt = c < n ? (c > 0 ? c : 0) : n;  // outputs hold n slots
    const int64_t warp =
        ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i0 = warp * 32; i0 < cnt; i0 += nwarps * 32) {
        const int np = (int)(cnt - i0 < 32 ? cnt - i0 : 32);
        const int64_t my_src = lane < np ? index[i0 + lane] : -1;
        const int total = np * w16;
        for (int t0 = 0; t0 < total; t0 += 32) {  // warp-uniform
            const int t = t0 + lane;
            const uint32_t tc = (uint32_t)(t < total ? t : total - 1);
            // the magic quotient is exact while tc * w16 < 2^32, i.e. for
            // w16 < 11585; longer sequences divide plainly
            const uint32_t p = w16 < 11585
                                   ? fast_div(tc, (uint32_t)w16, w16_magic)
                                   : tc / (uint32_t)w16;
            const int w = (int)(tc - p * (uint32_t)w16);
            const int64_t src = __shfl_sync(0xffffffffu, my_src, (int)p);
            if (t < total && src >= 0 && src < n) {
                const int64_t o = (i0 + p) * w16 + w;
                out_reads[o] = __ldg(reads + src * w16 + w);
                out_refs[o] = __ldg(refs + src * w16 + w);
            }
        }
    }
}

size_t compact_ws_bytes(int64_t n)
{
    return (size_t)((n + kCompactChunk - 1) / kCompactChunk + 1) * 8 + 256;
}

cudaError_t launch_compact(const uint8_t *acc, int64_t n, int64_t *ws,
                           int64_t *out_index, int64_t *out_count,
                           cudaStream_t st)
{
    if (n <= 0)
        return cudaMemsetAsync(out_count, 0, sizeof(int64_t), st);
    const int64_t nb = (n + kCompactChunk - 1) / kCompactChunk;
    if (nb > 0x7fffffff)
        return cudaErrorInvalidValue;
    k_compact_count<<<(unsigned)nb, kCompactThreads, 0, st>>>(acc, n, ws);
    k_compact_scan<<<1, 1024, 0, st>>>(ws, nb, out_count);
    k_compact_scatter<<<(unsigned)nb, kCompactThreads, 0, st>>>(acc, n, ws,
                                                                out_index);
    return cudaGetLastError();
}

cudaError_t launch_gather_pairs(const uint32_t *reads, const uint32_t *refs,
                                int32_t m, const int64_t *index,
                                const int64_t *count, int64_t n,
                                uint32_t *out_reads, uint32_t *out_refs,
                                int sm_count, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    const int w16 = (m + 15) / 16;
    if (w16 == 0)
        return cudaSuccess;
    k_gather_pairs<<<sm_count * 8, 256, 0, st>>>(
        reads, refs, w16, div_magic((uint32_t)w16), index, count, out_reads,
        out_refs, n);
    return cudaGetLastError();
}

}  // namespace ssk
