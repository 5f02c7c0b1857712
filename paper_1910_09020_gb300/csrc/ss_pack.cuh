// ss_pack.cuh -- the arithmetic of K1 (ASCII -> SS_FMT_PACKED2), shared by
// the fixed-stride and per-pair pack kernels.
//
// Eq. 1 only ever asks whether two bases are equal, so the filter works on a
// 2-bit code per base, A/C/G/T (either case) -> 0/1/2/3.  From bits b1..b3
// of the ASCII byte: code bit 0 = b1 ^ b2, code bit 1 = b2 ^ b3.
//
// Validity, per byte x (four per 32-bit lane op): the eight letters are
// exactly the bytes with d = (x & 0xD9) ^ 0x41 equal to 0x11 * (b2 & ~b1):
// bits 7, 3 clear and bit 6 set for all of them; bits 0 and 4 read 1, 0
// for a/c/g (b2 b1 != 10) and 0, 1 for t (b2 b1 = 10); bit 5 (case), b1
// and b2 are free.  The test suite checks this rule on all 256 byte values.
#pragma once
#include <cstdint>

#include "ss_device.cuh"

namespace ssk {

// 16 ASCII bytes (x[q] holds bytes 4q..4q+3, little-endian) -> one packed
// word (bit j = code bit 0 of byte j, bit 16+j = code bit 1).  err gets a
// nonzero bit for every byte that is not a base.
//
// Gather: k0 holds code bit 0 of byte i at bit 8i+1; two words combine into
// bits 8i+1 and 8i+5, and one multiply by 2^23 + 2^16 + 2^9 + 2^2 moves
// bit 8i+1 to 24+i and bit 8i+5 to 28+i.  Every other partial product lands
// on a distinct bit below 24 or above 31, so no carry reaches bits 24..31.
SS_HD uint32_t pack_chunk(const uint32_t x[4], uint32_t &err)
{
    uint32_t k0[4], k1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t f = x[q] >> 1;
        const uint32_t y = x[q] ^ f;
        k0[q] = y & 0x02020202u;
        k1[q] = y & 0x04040404u;
        const uint32_t t = (x[q] >> 2) & ~f & 0x01010101u;  // b2 & ~b1
        const uint32_t d = (x[q] & 0xD9D9D9D9u) ^ 0x41414141u;
        err |= d ^ (t * 17u);
    }
    const uint32_t lo01 = (k0[1] * 16u + k0[0]) * 0x00810204u;
    const uint32_t lo23 = (k0[3] * 16u + k0[2]) * 0x00810204u;
    const uint32_t hi01 = (k1[1] * 16u + k1[0]) * 0x00408102u;
    const uint32_t hi23 = (k1[3] * 16u + k1[2]) * 0x00408102u;
    return prmt(prmt(lo01, lo23, 0x73u), prmt(hi01, hi23, 0x73u), 0x5410u);
}

// 16 ASCII bytes -> their 32 code bits in base order, base t's code at bits
// 2t (code bit 0) and 2t+1 (code bit 1); err as above.  Word x[q] holds
// bases 4q..4q+3: y = (x ^ x >> 1) & 0x06060606 keeps, for byte i, code bit
// 0 at bit 8i+1 and code bit 1 at 8i+2, and one multiply by 2^23 + 2^17 +
// 2^11 + 2^5 moves them to bits 24+2i and 25+2i.  Its partial products, bit
// 8i+1+b times 2^(23-6k), land at 24 + 8i - 6k + b, distinct for all i, k
// in 0..3 and b in 0..1, so nothing carries; the top bytes of the four
// products are the four bytes of the result.
SS_HD uint32_t pack_chunk_pairs(const uint32_t x[4], uint32_t &err)
{
    uint32_t p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t f = x[q] >> 1;
        const uint32_t y = (x[q] ^ f) & 0x06060606u;
        p[q] = y * 0x00820820u;
        const uint32_t t = (x[q] >> 2) & ~f & 0x01010101u;  // b2 & ~b1
        const uint32_t d = (x[q] & 0xD9D9D9D9u) ^ 0x41414141u;
        err |= d ^ (t * 17u);
    }
    return prmt(prmt(p[0], p[1], 0x0073u), prmt(p[2], p[3], 0x0073u),
                0x5410u);
}

// 16 codes starting at base r (0..15) of two consecutive packed words c0, c1
// of one base stream.
SS_HD uint32_t pack_window(uint32_t c0, uint32_t c1, uint32_t r)
{
    const uint32_t lo = prmt(c0, c1, 0x5410u) >> r;
    const uint32_t hi = prmt(c0, c1, 0x7632u) >> r;
    return prmt(lo, hi, 0x5410u);
}

}  // namespace ssk
