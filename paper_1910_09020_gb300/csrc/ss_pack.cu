// ss_pack.cu -- K1: ASCII bases -> SS_FMT_PACKED2 (2 bits per base).
//
// Eq. 1 only ever asks whether two bases are equal, so the filter works on a
// 2-bit code of each base.  The code is computed arithmetically from the
// ASCII byte: with v = byte | 0x20 (lower case), bit 0 = bit1(v) ^ bit2(v)
// and bit 1 = bit2(v) ^ bit3(v), which maps a/c/g/t to 0/1/2/3.  A byte is
// valid iff v equals the canonical letter of its code; anything else latches
// kStatusInvalidBase.  Four bytes are handled per 32-bit lane operation.
//
// One thread writes one output word (16 bases); the kernel is bound by HBM
// bandwidth (16 bytes read, 4 written per word).
#include <cstdint>

#include "ss_device.cuh"
#include "ss_internal.h"

namespace ssk {

// Four ASCII bytes -> 4 code-bit-0 bits, 4 code-bit-1 bits; false if any
// byte is not a base.  Missing bytes must be passed as 'A'.  With
// y = x ^ (x >> 1), code bit 0 = y bit 1 and code bit 1 = y bit 2 of every
// byte (bit 5, the case bit, does not enter), so one shift and one XOR
// serve both bits.
__device__ __forceinline__ bool codes4(uint32_t x, uint32_t &lo4,
                                       uint32_t &hi4)
{
    const uint32_t y = x ^ (x >> 1);
    const uint32_t k0 = (y >> 1) & 0x01010101u;
    const uint32_t k1 = (y >> 2) & 0x01010101u;
    // gather bits 0, 8, 16, 24 into bits 0..3 (no carries can occur)
    lo4 = (k0 * 0x10204080u) >> 28;
    hi4 = (k1 * 0x10204080u) >> 28;
    // canonical lower-case letter per code: 'a' + {0, 2, 6, 19}[code]
    const uint32_t canon =
        0x61616161u + k0 * 2u + k1 * 6u + (k0 & k1) * 11u;
    return (x | 0x20202020u) == canon;
}

// Pack up to 16 bases starting at src (len in 1..16).
__device__ __forceinline__ uint32_t pack16(const uint8_t *__restrict__ src,
                                           int len, bool aligned4,
                                           bool &valid)
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
    uint32_t lo = 0, hi = 0;
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t l4, h4;
        ok &= codes4(w[q], l4, h4);
        lo |= l4 << (4 * q);
        hi |= h4 << (4 * q);
    }
    valid = ok;
    return lo | (hi << 16);
}

// Fixed stride: pair p at byte p*m, output at word p*w16.  A CTA writes
// kPackWords consecutive output words; the ASCII bytes behind them are one
// contiguous span, which the CTA first copies to shared memory with 16-byte
// loads (every thread keeps several loads in flight), then each thread builds
// its words from shared memory.
constexpr int kPackThreads = 256;
constexpr int kPackWords = 1024;  // output words per CTA (4 per thread)
constexpr int kPackSpan = kPackWords * 16 + 32;  // staged bytes, with slack

__global__ void __launch_bounds__(kPackThreads)
    k_pack_fixed(const uint8_t *__restrict__ ascii, int64_t n, int32_t m,
                 int32_t w16, uint32_t w16_magic, uint32_t *__restrict__ out,
                 int *status)
{
    __shared__ __align__(16) uint8_t span[kPackSpan];
    const int64_t total = n * (int64_t)w16;
    const int64_t g0 = (int64_t)blockIdx.x * kPackWords;
    if (g0 >= total)
        return;
    const int64_t g1 = min(g0 + (int64_t)kPackWords, total);  // exclusive
    const int64_t pa = g0 / w16;
    const int wa = (int)(g0 - pa * w16);
    const int64_t pb = (g1 - 1) / w16;
    const int wb = (int)(g1 - 1 - pb * w16);
    const int64_t b0 = pa * m + 16 * (int64_t)wa;             // first byte
    const int64_t b1 = pb * m + min(16 * (wb + 1), m);         // end byte
    const int64_t base = b0 & ~(int64_t)15;
    const int64_t limit = n * (int64_t)m;                      // input size
    // stage [base, b1) -- full 16-byte chunks inside the input, bytes else
    const int chunks = (int)((b1 - base + 15) >> 4);
    const uint4 *src = reinterpret_cast<const uint4 *>(ascii + base);
    uint4 *dst = reinterpret_cast<uint4 *>(span);
    const bool aligned = ((uintptr_t)ascii & 15) == 0;
    for (int c = threadIdx.x; c < chunks; c += kPackThreads) {
        const int64_t at = base + 16 * (int64_t)c;
        if (aligned && at + 16 <= limit) {
            dst[c] = __ldg(src + c);
        } else {
            for (int k = 0; k < 16; ++k)
                span[16 * c + k] = at + k < limit ? __ldg(ascii + at + k)
                                                  : (uint8_t)0x41;
        }
    }
    __syncthreads();
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(span);
    bool bad = false;
    // byte offset in the span of the CTA's first pair
    const int off0 = (int)(pa * m - base);
#pragma unroll
    for (int k = 0; k < kPackWords / kPackThreads; ++k) {
        const int j = k * kPackThreads + threadIdx.x;
        if (g0 + j < g1) {
            // pair (relative to the CTA's first) and word of output g0 + j
            const uint32_t rel = (uint32_t)wa + (uint32_t)j;
            const uint32_t dp = fast_div(rel, (uint32_t)w16, w16_magic);
            const int w = (int)(rel - dp * (uint32_t)w16);
            const int off = off0 + (int)dp * m + 16 * w;
            const int len = m - 16 * w;  // >= 16 except on a pair's last word
            const int a = off >> 2;
            const uint32_t sh = (uint32_t)(off & 3) * 8u;
            uint32_t x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                x[q] = funnel_r(s32[a + q], s32[a + q + 1], sh);
            if (len < 16) {
                // bytes past the sequence's end count as 'A' (code 0)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int keep = len - 4 * q;
                    const uint32_t km =
                        keep <= 0 ? 0u
                                  : (keep >= 4 ? 0xffffffffu
                                               : (0xffffffffu >> (32 - 8 * keep)));
                    x[q] = (x[q] & km) | (0x41414141u & ~km);
                }
            }
            uint32_t lo = 0, hi = 0;
            bool ok = true;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t l4, h4;
                ok &= codes4(x[q], l4, h4);
                lo += l4 << (4 * q);
                hi += h4 << (4 * q);
            }
            out[g0 + j] = lo | (hi << 16);
            bad |= !ok;
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
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
        bool pair_bad = false;
        for (int w = lane; w < w16; w += 32) {
            const uint8_t *s = src + (int64_t)w * 16;
            const int len = min(16, m - w * 16);
            bool valid;
            dst[w] = pack16(s, len, ((uintptr_t)s & 3) == 0, valid);
            pair_bad |= !valid;
        }
        pair_bad = __any_sync(0xffffffffu, pair_bad);
        if (pair_bad && bad_flags && lane == 0)
            bad_flags[p] = 1;
        any_bad |= pair_bad;
    }
    if (any_bad && lane == 0)
        atomicOr(status, kStatusInvalidBase);
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
