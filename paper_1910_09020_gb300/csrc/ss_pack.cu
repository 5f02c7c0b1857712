// ss_pack.cu -- K1: ASCII bases -> SS_FMT_PACKED2 (2 bits per base).
//
// The code arithmetic and the validity rule are in ss_pack.cuh.  A byte that
// is not A/C/G/T (either case) latches kStatusInvalidBase.
//
// Fixed-stride kernel: the CTA owns kPackWords consecutive output words,
// whose ASCII bytes form one contiguous span of the input.  Phase 1 reads
// that span as aligned 16-byte chunks (one coalesced 128-bit load each, all
// of a thread's loads in flight together) and turns every chunk into one
// packed word of a "code stream" in shared memory.  Phase 2 builds each
// output word -- 16 codes starting at its pair's base 16w -- as a window of
// two consecutive code-stream words, and zeroes the codes past the pair's
// end.  The kernel is bound by HBM bandwidth (m bytes read, 4 * ceil(m/16)
// written per sequence).
#include <algorithm>
#include <cstdint>

#include "ss_device.cuh"
#include "ss_internal.h"
#include "ss_pack.cuh"
#include "ss_sliced.cuh"

namespace ssk {

// Pack up to 16 bases starting at src (len in 1..16); bytes past len count
// as 'A' (code 0).
__device__ __forceinline__ uint32_t pack16(const uint8_t *__restrict__ src,
                                           int len, bool aligned4,
                                           uint32_t &err)
{
    uint32_t w[4];
    if (len == 16 && aligned4) {
        const uint32_t *s4 = reinterpret_cast<const uint32_t *>(src);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            w[q] = __ldg(s4 + q);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t x = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int j = q * 4 + b;
                const uint32_t c = j < len ? (uint32_t)__ldg(src + j) : 0x41u;
                x |= c << (8 * b);
            }
            w[q] = x;
        }
    }
    return pack_chunk(w, err);
}

constexpr int kPackThreads = 256;
constexpr int kPackWords = 1024;             // output words per CTA
constexpr int kPackChunks = kPackWords + 4;  // code-stream words per CTA
constexpr int kPackIter = (kPackChunks + kPackThreads - 1) / kPackThreads;

// Fixed stride: pair p at byte p*m, output at word p*w16.
__global__ void __launch_bounds__(kPackThreads, 8)
    k_pack_fixed(const uint8_t *__restrict__ ascii, int64_t n, int32_t m,
                 int32_t w16, uint32_t w16_magic, uint32_t *__restrict__ out,
                 int *status)
{
    __shared__ uint32_t code[kPackChunks];
    __shared__ int64_t s_pair[2];
    const int64_t total = n * (int64_t)w16;
    const int64_t g0 = (int64_t)blockIdx.x * kPackWords;
    if (g0 >= total)
        return;
    const int64_t g1 = min(g0 + (int64_t)kPackWords, total);  // exclusive
    // the pairs of the first and last word: two 64-bit divisions, done by
    // one thread (each costs a warp tens of instructions)
    if (threadIdx.x == 0) {
        s_pair[0] = g0 / w16;
        s_pair[1] = (g1 - 1) / w16;
    }
    __syncthreads();
    const int64_t pa = s_pair[0];
    const int wa = (int)(g0 - pa * w16);
    const int64_t pb = s_pair[1];
    const int wb = (int)(g1 - 1 - pb * w16);
    const int64_t b0 = pa * m + 16 * (int64_t)wa;      // first byte
    const int64_t b1 = pb * m + min(16 * (wb + 1), m);  // end byte
    const int64_t cb = b0 >> 4;                        // first chunk
    // chunks [cb, cb + nc): the span, plus one (windows read chunk k+1)
    const int nc = (int)(((b1 + 15) >> 4) - cb) + 1;
    const int64_t limit = n * (int64_t)m;  // input bytes
    // every chunk of the span whole, 16-byte aligned and inside the input:
    // the common case, one uniform branch for the CTA
    const bool fast = ((uintptr_t)ascii & 15) == 0 &&
                      (cb + nc) * 16 <= limit;
    uint32_t err = 0;
    // phase 1: chunks -> code stream
    uint32_t x[kPackIter][4];
    if (fast) {
        const uint4 *src = reinterpret_cast<const uint4 *>(ascii) + cb;
#pragma unroll
        for (int i = 0; i < kPackIter; ++i) {
            const int c = (int)threadIdx.x + i * kPackThreads;
            if (c < nc) {
                const uint4 v = __ldg(src + c);
                x[i][0] = v.x;
                x[i][1] = v.y;
                x[i][2] = v.z;
                x[i][3] = v.w;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < kPackIter; ++i) {
            const int c = (int)threadIdx.x + i * kPackThreads;
            const int64_t at = (cb + c) * 16;
            if (c < nc) {
                if (((uintptr_t)ascii & 15) == 0 && at + 16 <= limit) {
                    const uint4 v =
                        __ldg(reinterpret_cast<const uint4 *>(ascii + at));
                    x[i][0] = v.x;
                    x[i][1] = v.y;
                    x[i][2] = v.z;
                    x[i][3] = v.w;
                } else {
                    // the input's last partial chunk, or an unaligned input:
                    // bytes past the end count as 'A'
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t w = 0;
                        for (int b = 0; b < 4; ++b) {
                            const int64_t j = at + 4 * q + b;
                            const uint32_t ch =
                                j < limit ? (uint32_t)__ldg(ascii + j) : 0x41u;
                            w |= ch << (8 * b);
                        }
                        x[i][q] = w;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kPackIter; ++i) {
        const int c = (int)threadIdx.x + i * kPackThreads;
        if (c < nc)
            code[c] = pack_chunk(x[i], err);
    }
    __syncthreads();
    // phase 2: output word (pair pa + dp, word w) starts at stream byte
    // o = (pa + dp) * m + 16 w - 16 cb
    const uint32_t o0 = (uint32_t)(pa * m - cb * 16);
#pragma unroll
    for (int k = 0; k < kPackWords / kPackThreads; ++k) {
        const int j = k * kPackThreads + (int)threadIdx.x;
        if (g0 + j < g1) {
            const uint32_t rel = (uint32_t)wa + (uint32_t)j;
            const uint32_t dp = fast_div(rel, (uint32_t)w16, w16_magic);
            const uint32_t w = rel - dp * (uint32_t)w16;
            const uint32_t o = o0 + dp * (uint32_t)m + 16u * w;
            const uint32_t kk = o >> 4;
            const uint32_t v = pack_window(code[kk], code[kk + 1], o & 15u);
            // codes past the pair's end (its last word) are zero, no branch
            const uint32_t keep = mask_below(m - 16 * (int)w) & 0xffffu;
            out[g0 + j] = v & (keep * 0x10001u);
        }
    }
    if (__any_sync(0xffffffffu, err != 0u) && (threadIdx.x & 31) == 0)
        atomicOr(status, kStatusInvalidBase);
}

// Per-pair offsets and lengths: one warp per pair, lanes over its words.
// bad (optional): per-pair flag set to 1 when the pair holds a non-base.
__global__ void k_pack_varlen(const uint8_t *__restrict__ ascii,
                              const int64_t *__restrict__ offsets,
                              const int32_t *__restrict__ lengths, int64_t n,
                              uint32_t *__restrict__ out,
                              const int64_t *__restrict__ out_offsets,
                              int *status, uint8_t *bad_flags)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool any_bad = false;
    for (int64_t p = warp; p < n; p += nwarps) {
        const int32_t m = lengths[p];
        if (m <= 0)
            continue;
        const uint8_t *src = ascii + offsets[p];
        uint32_t *dst = out + out_offsets[p];
        const int w16 = (m + 15) >> 4;
        uint32_t err = 0;
        for (int w = lane; w < w16; w += 32) {
            const uint8_t *s = src + (int64_t)w * 16;
            const int len = min(16, m - w * 16);
            dst[w] = pack16(s, len, ((uintptr_t)s & 3) == 0, err);
        }
        bool pair_bad = err != 0u;
        pair_bad = __any_sync(0xffffffffu, pair_bad);
        if (pair_bad && bad_flags && lane == 0)
            bad_flags[p] = 1;
        any_bad |= pair_bad;
    }
    if (any_bad && lane == 0)
        atomicOr(status, kStatusInvalidBase);
}

// Fixed stride -> the bit-sliced layout (SS_FMT_SLICED2): one warp per
// group of 32 pairs.  Lane i packs 16 bases of pair 32g + i into one word
// (bit t = code bit 0 of base t, bit 16 + t = code bit 1); the warp then
// transposes the 32 words (lanes x bits), so lane r holds code bit r/16 of
// base r%16 of all 32 pairs, which is one word of the layout.
constexpr int kPackSlicedWarps = 8;

__device__ __forceinline__ uint32_t warp_transpose32(uint32_t v, int lane)
{
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const uint32_t x = __shfl_xor_sync(0xffffffffu, v, d);
        v = transpose_level(v, x, lane, d);
    }
    return v;
}

// The same transpose with its per-lane constants computed once per thread
// (transpose_level's byte selectors, rotations and masks for this lane).
struct LaneTranspose {
    uint32_t s16, s8, a4, a2, a1, k4, k2, k1;
    __device__ __forceinline__ explicit LaneTranspose(int lane)
    {
        s16 = (lane & 16) ? 0x3276u : 0x5410u;
        s8 = (lane & 8) ? 0x3715u : 0x6240u;
        a4 = (lane & 4) ? 28u : 4u;
        a2 = (lane & 2) ? 30u : 2u;
        a1 = (lane & 1) ? 31u : 1u;
        k4 = (lane & 4) ? 0xf0f0f0f0u : 0x0f0f0f0fu;
        k2 = (lane & 2) ? 0xccccccccu : 0x33333333u;
        k1 = (lane & 1) ? 0xaaaaaaaau : 0x55555555u;
    }
    // (v & k) | (rotl(x, a) & ~k): one rotate and one lop3 per level
    __device__ __forceinline__ static uint32_t level(uint32_t v, uint32_t x,
                                                     uint32_t a, uint32_t k)
    {
        return lop3<0xE4>(v, funnel_l(x, x, a), k);
    }
    __device__ __forceinline__ uint32_t operator()(uint32_t v) const
    {
        uint32_t x = __shfl_xor_sync(0xffffffffu, v, 16);
        v = prmt(v, x, s16);
        x = __shfl_xor_sync(0xffffffffu, v, 8);
        v = prmt(v, x, s8);
        x = __shfl_xor_sync(0xffffffffu, v, 4);
        v = level(v, x, a4, k4);
        x = __shfl_xor_sync(0xffffffffu, v, 2);
        v = level(v, x, a2, k2);
        x = __shfl_xor_sync(0xffffffffu, v, 1);
        return level(v, x, a1, k1);
    }
};

__global__ void __launch_bounds__(32 * kPackSlicedWarps)
    k_pack_sliced(const uint8_t *__restrict__ ascii, int64_t n, int32_t m,
                  int64_t G, uint32_t *__restrict__ out, int *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t g =
        (int64_t)blockIdx.x * kPackSlicedWarps + (threadIdx.x >> 5);
    if (g >= G)
        return;  // the whole warp
    const int64_t p = g * 32 + lane;
    const bool live = p < n;
    const uint8_t *src = ascii + (live ? p : 0) * (int64_t)m;
    const bool aligned4 = ((uintptr_t)src & 3) == 0;
    const int w16 = (m + 15) >> 4;
    const int nb4 = 4 * ((m + 3) >> 2);  // bases of the stored blocks
    uint32_t err = 0;
    for (int c = 0; c < w16; ++c) {
        uint32_t w = 0u;
        if (live)
            w = pack16(src + 16 * c, min(16, m - 16 * c), aligned4, err);
        w = warp_transpose32(w, lane);
        const int j = 16 * c + (lane & 15);
        if (j < nb4)
            out[((int64_t)(j >> 2) * G + g) * 8 + (lane >> 4) * 4 + (j & 3)] =
                w;
    }
    if (__any_sync(0xffffffffu, err != 0u) && lane == 0)
        atomicOr(status, kStatusInvalidBase);
}

// Two-phase form for reads up to kPackSpanMaxM bases: a CTA's groups (gpc of
// them, 32 gpc consecutive pairs) are one contiguous span of the input.
// Phase 1 reads the span as aligned 16-byte chunks, coalesced, and turns
// each into one word of a code stream in shared memory (pack_chunk_pairs:
// the chunk's base t at bits 2t and 2t+1).  Phase 2 gives each lane its
// pair's 16-base windows, one funnel shift of two consecutive stream words
// each, with the codes past the pair's end cleared, and the warp transposes
// them as above (lane r then holds code bit r%2 of base r/2).
constexpr int kPackSpanMaxWords = 12 * 1024;  // 48 KB of code stream
// 8 CTAs of 256 threads per SM (32 registers): the load phase of one CTA
// overlaps the transpose phase of the others (measured 0.75 -> 0.69 ms per
// 30M x 100 bp side against the compiler's 40 registers, 6 CTAs)
constexpr int kPackSpanMaxM = (kPackSpanMaxWords - 3) / 2;

__global__ void __launch_bounds__(32 * kPackSlicedWarps, 8)
    k_pack_sliced_span(const uint8_t *__restrict__ ascii, int64_t n,
                       int32_t m, int64_t G, int gpc,
                       uint32_t *__restrict__ out, int *status)
{
    extern __shared__ uint32_t code[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t g0 = (int64_t)blockIdx.x * gpc;
    const int64_t p0 = g0 * 32;
    const int64_t p1 = min(n, p0 + 32 * (int64_t)gpc);  // pairs [p0, p1)
    const int64_t cb = (p0 * m) >> 4;                   // first chunk
    // chunks [cb, cb + nc): the span, plus one (windows read word k+1)
    const int nc = (int)(((p1 * m + 15) >> 4) - cb) + 1;
    const int64_t limit = n * (int64_t)m;
    // every chunk whole, 16-byte aligned and inside the input: the common
    // case, one uniform branch for the CTA
    const bool fast =
        ((uintptr_t)ascii & 15) == 0 && (cb + nc) * 16 <= limit;
    uint32_t err = 0;
    if (fast) {
        // four loads of a thread in flight before any is packed (0.69 ->
        // 0.66 ms per 30M x 100 bp side with the full-group branch below)
        const uint4 *src = reinterpret_cast<const uint4 *>(ascii) + cb;
        constexpr int T = 32 * kPackSlicedWarps;
        for (int c0 = threadIdx.x; c0 < nc; c0 += 4 * T) {
            uint4 v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (c0 + i * T < nc)
                    v[i] = __ldg(src + c0 + i * T);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (c0 + i * T < nc) {
                    const uint32_t x[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
                    code[c0 + i * T] = pack_chunk_pairs(x, err);
                }
        }
    } else {
        for (int c = threadIdx.x; c < nc; c += 32 * kPackSlicedWarps) {
            const int64_t at = (cb + c) * 16;
            uint32_t x[4];
            if (((uintptr_t)ascii & 15) == 0 && at + 16 <= limit) {
                const uint4 v =
                    __ldg(reinterpret_cast<const uint4 *>(ascii + at));
                x[0] = v.x;
                x[1] = v.y;
                x[2] = v.z;
                x[3] = v.w;
            } else {
                // the input's last partial chunk, or an unaligned input:
                // bytes past the end count as 'A'
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t w = 0;
                    for (int b = 0; b < 4; ++b) {
                        const int64_t j = at + 4 * q + b;
                        const uint32_t ch =
                            j < limit ? (uint32_t)__ldg(ascii + j) : 0x41u;
                        w |= ch << (8 * b);
                    }
                    x[q] = w;
                }
            }
            code[c] = pack_chunk_pairs(x, err);
        }
    }
    __syncthreads();
    const int64_t g = g0 + warp;
    if (warp < gpc && g < G) {
        const int64_t p = g * 32 + lane;
        const uint32_t live = p < n ? 0xffffffffu : 0u;
        const int w16 = (m + 15) >> 4;
        const LaneTranspose tr(lane);
        // bit of the stream where the pair's base 0 sits (pad lanes read
        // the group's first pair and keep nothing): its 16-base windows are
        // one funnel shift by o0 % 32 of stream words o0/32 + c, + c + 1
        const uint32_t o0 =
            (uint32_t)(2 * ((p < n ? p : g * 32) * m - cb * 16));
        const uint32_t sh = o0 & 31u;
        const uint32_t *src = code + (o0 >> 5);
        // lane r stores code bit r%2 of base 16c + r/2: word
        // ((4c + r/8) * G + g) * 8 + (r%2) * 4 + (r/2)%4
        uint32_t *dst = out + ((int64_t)(lane >> 3) * G + g) * 8 +
                        (lane & 1) * 4 + ((lane >> 1) & 3);
        const int64_t step = 32 * G;  // four blocks
        uint32_t cur = src[0];
        if ((g + 1) * 32 <= n) {  // a full group: every lane a pair
            for (int c = 0; c + 1 < w16; ++c) {
                const uint32_t nxt = src[c + 1];
                dst[c * step] = tr(funnel_r(cur, nxt, sh));
                cur = nxt;
            }
        } else {
            for (int c = 0; c + 1 < w16; ++c) {
                const uint32_t nxt = src[c + 1];
                dst[c * step] = tr(funnel_r(cur, nxt, sh) & live);
                cur = nxt;
            }
        }
        // the last 16 bases: codes past the pair's end cleared, words of
        // blocks past the last one not stored
        const int c = w16 - 1;
        const uint32_t w = tr(funnel_r(cur, src[c + 1], sh) & live &
                              mask_below(2 * (m - 16 * c)));
        if (16 * c + (lane >> 1) < 4 * ((m + 3) >> 2))
            dst[c * step] = w;
    }
    if (__any_sync(0xffffffffu, err != 0u) && lane == 0)
        atomicOr(status, kStatusInvalidBase);
}

cudaError_t launch_pack_sliced(const uint8_t *ascii, int64_t n, int32_t m,
                               uint32_t *out, int *status, cudaStream_t st)
{
    if (n <= 0 || m <= 0)
        return cudaSuccess;
    const int64_t G = (n + 31) / 32;
    if (m <= kPackSpanMaxM) {
        // groups per CTA: as many as the warps, while the span's code
        // stream fits
        const int gpc = (int)std::min<int64_t>(
            kPackSlicedWarps, (kPackSpanMaxWords - 3) / (2 * (int64_t)m));
        const int64_t blocks = (G + gpc - 1) / gpc;
        if (blocks > 0x7fffffff)
            return cudaErrorInvalidValue;
        const size_t smem = ((size_t)2 * gpc * m + 3) * 4;
        k_pack_sliced_span<<<(unsigned)blocks, 32 * kPackSlicedWarps, smem,
                             st>>>(ascii, n, m, G, gpc, out, status);
        return cudaGetLastError();
    }
    const int64_t blocks = (G + kPackSlicedWarps - 1) / kPackSlicedWarps;
    if (blocks > 0x7fffffff)
        return cudaErrorInvalidValue;
    k_pack_sliced<<<(unsigned)blocks, 32 * kPackSlicedWarps, 0, st>>>(
        ascii, n, m, G, out, status);
    return cudaGetLastError();
}

cudaError_t launch_pack_fixed(const uint8_t *ascii, int64_t n, int32_t m,
                              uint32_t *out, int *status, cudaStream_t st)
{
    if (n <= 0 || m <= 0)
        return cudaSuccess;
    const int32_t w16 = (m + 15) / 16;
    const int64_t total = n * (int64_t)w16;
    const int64_t blocks = (total + kPackWords - 1) / kPackWords;
    if (blocks > 0x7fffffff)
        return cudaErrorInvalidValue;
    k_pack_fixed<<<(unsigned)blocks, kPackThreads, 0, st>>>(
        ascii, n, m, w16, div_magic((uint32_t)w16), out, status);
    return cudaGetLastError();
}

cudaError_t launch_pack_varlen(const uint8_t *ascii, const int64_t *offsets,
                               const int32_t *lengths, int64_t n,
                               uint32_t *out, const int64_t *out_offsets,
                               int *status, int sm_count, cudaStream_t st,
                               uint8_t *bad_flags)
{
    if (n <= 0)
        return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (n * 32 + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count * 8;
    if (blocks > cap)
        blocks = cap;
    k_pack_varlen<<<(unsigned)blocks, threads, 0, st>>>(
        ascii, offsets, lengths, n, out, out_offsets, status, bad_flags);
    return cudaGetLastError();
}

}  // namespace ssk
