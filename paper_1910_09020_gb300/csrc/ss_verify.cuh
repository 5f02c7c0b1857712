// ss_verify.cuh -- the accuracy harness: exact edit distance (up to E+1) of
// read/reference pairs on the GPU, to measure the filter's false accept and
// false reject rates the way Section 3.2 does with an aligner as ground truth.
//
// Banded Levenshtein DP (Ukkonen): any alignment of cost <= E stays within
// |i - j| <= E, so evaluating only the 2E+1 diagonals of each row and
// saturating at E+1 gives min(ED, E+1) exactly.  One thread per pair; the
// band of the previous row lives in registers (E <= 31 is a template
// parameter);
// the mismatches of a whole band row come from one comparison of a window
// of the reference's bit planes with the read base broadcast.
#pragma once
#include <cstdint>

#include "ss_device.cuh"

namespace ssk {

struct EdArgs {
    const uint32_t *reads;  // packed, pair p at word p * w16
    const uint32_t *refs;
    int64_t n;
    int32_t m;
    int32_t w16;
    int32_t *ed;            // out: min(ED, E+1)
};

// Bit t of the result = code bit (plane 0 or 1) of base pos + t of a packed
// sequence, for t in 0..63; zero outside 0..m-1.  pos may be negative.
SS_HD uint64_t plane_window(const uint32_t *g, int w16, int m, int pos,
                            int plane)
{
    uint64_t out = 0;
    // five packed words (16 bases each) cover any 64 positions
    const int first = pos >= 0 ? pos >> 4 : -((15 - pos) >> 4);
    for (int k = 0; k < 5; ++k) {
        const int wi = first + k;
        if (wi < 0 || wi >= w16)
            continue;
        const uint32_t word = ldg(g + wi);
        uint64_t bits = plane ? (word >> 16) : (word & 0xffffu);
        const int start = wi * 16;  // position of bit 0 of `bits`
        const int valid = m - start < 16 ? m - start : 16;
        if (valid < 16)
            bits &= (1ull << valid) - 1ull;
        const int sh = start - pos;
        if (sh >= 64 || sh <= -16)
            continue;
        out |= sh >= 0 ? bits << sh : bits >> -sh;
    }
    return out;
}

template <int E>
SS_HD int ed_banded(const uint32_t *q, const uint32_t *r, int m, int w16)
{
    constexpr int B = 2 * E + 1;  // band cells d = j - i + E, j in i-E..i+E
    constexpr int CAP = E + 1;
    int D[B];
    // row i = 0: D[0][j] = j for j in 0..E (d = j + E), outside = CAP
#pragma unroll
    for (int d = 0; d < B; ++d) {
        const int j = d - E;
        D[d] = (j >= 0 && j <= m) ? (j < CAP ? j : CAP) : CAP;
    }
    for (int i = 1; i <= m; ++i) {
        // read base i-1 (codes), reference window R[i-1-E .. i-1+E]
        const int qi = i - 1;
        const uint32_t qw = ldg(q + (qi >> 4));
        const uint32_t qlo = (qw >> (qi & 15)) & 1u;
        const uint32_t qhi = (qw >> (16 + (qi & 15))) & 1u;
        const int pos = i - 1 - E;  // reference index of band cell d = 0
        const uint64_t rlo = plane_window(r, w16, m, pos, 0);
        const uint64_t rhi = plane_window(r, w16, m, pos, 1);
        const uint64_t mm = (rlo ^ (0ull - (uint64_t)qlo)) |
                            (rhi ^ (0ull - (uint64_t)qhi));  // 1 = mismatch
        int left = CAP;  // D[i][j-1] of the cell being computed
#pragma unroll
        for (int d = 0; d < B; ++d) {
            const int j = i + d - E;
            int v;
            if (j < 0 || j > m) {
                v = CAP;
            } else if (j == 0) {
                v = i < CAP ? i : CAP;
            } else {
                const int diag = D[d] + (int)((mm >> d) & 1ull);
                const int up = (d + 1 < B ? D[d + 1] : CAP) + 1;
                v = diag < up ? diag : up;
                v = v < left + 1 ? v : left + 1;
                v = v < CAP ? v : CAP;
            }
            D[d] = v;
            left = v;
        }
    }
    return D[E];  // j = i = m
}

}  // namespace ssk
