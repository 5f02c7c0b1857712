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

// ---- large thresholds: one warp per pair -----------------------------------
//
// The same banded DP for E up to 511: the 2E+1 band cells of a row are
// spread over the 32 lanes, C consecutive cells per lane, in registers.  The
// in-row dependency D[i][j] = min(T[j], D[i][j-1] + 1), with T the best of
// the diagonal and upper neighbours, is a prefix minimum: D[d] = d +
// min_{d' <= d} (T[d'] - d'), computed per lane and then across the warp
// with shuffles.  The reference bases of a lane's cells come from a 64-base
// window of its bit planes, re-read every 32 rows.  Once every cell of a
// row exceeds E, ED > E (every alignment passes through that row).
template <int C>
__device__ int ed_band_warp(const uint32_t *q, const uint32_t *r, int m,
                            int E)
{
    const int lane = threadIdx.x & 31;
    const int B = 2 * E + 1;
    const int CAP = E + 1;
    const int BIG = 1 << 30;
    const int w16 = (m + 15) >> 4;
    int P[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {  // row 0: D[0][j] = j
        const int d = lane * C + c, j = d - E;
        P[c] = (d < B && j >= 0 && j <= m) ? (j < CAP ? j : CAP) : CAP;
    }
    uint64_t wlo = 0, whi = 0;
    int wstart = 0;
    for (int i = 1; i <= m; ++i) {
        const int b0 = i - E - 1 + lane * C;  // reference base of cell c = 0
        if (((i - 1) & 31) == 0) {            // warp-uniform refill
            wlo = plane_window(r, w16, m, b0, 0);
            whi = plane_window(r, w16, m, b0, 1);
            wstart = b0;
        }
        const int sh = b0 - wstart;           // 0..31
        const uint32_t qw = ldg(q + ((i - 1) >> 4));
        const uint64_t qlo = 0ull - (uint64_t)((qw >> ((i - 1) & 15)) & 1u);
        const uint64_t qhi =
            0ull - (uint64_t)((qw >> (16 + ((i - 1) & 15))) & 1u);
        const uint64_t mm = ((wlo >> sh) ^ qlo) | ((whi >> sh) ^ qhi);
        const int next0 = __shfl_down_sync(0xffffffffu, P[0], 1);
        int PM[C];
        int pm = BIG;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int d = lane * C + c, j = i + d - E;
            int up = c + 1 < C ? P[c + 1] : (lane < 31 ? next0 : CAP);
            if (d + 1 >= B)
                up = CAP;
            int t = P[c] + (int)((mm >> c) & 1ull);
            t = t < up + 1 ? t : up + 1;
            if (j == 0)
                t = i;                        // D[i][0] = i
            if (d >= B || j < 0 || j > m)
                t = CAP;
            const int u = t - d;
            pm = pm < u ? pm : u;
            PM[c] = pm;
        }
        // exclusive prefix minimum of the lanes' minima
        int incl = pm;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off)
                incl = incl < v ? incl : v;
        }
        int ex = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0)
            ex = BIG;
        int rowmin = CAP;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int d = lane * C + c, j = i + d - E;
            int v = d + (ex < PM[c] ? ex : PM[c]);
            v = v < CAP ? v : CAP;
            if (d >= B || j < 0 || j > m)
                v = CAP;
            P[c] = v;
            rowmin = rowmin < v ? rowmin : v;
        }
        if ((i & 7) == 0 &&
            __reduce_min_sync(0xffffffffu, (unsigned)rowmin) >= (unsigned)CAP)
            return CAP;
    }
    // cell d = E (j = i = m)
    int out = CAP;
#pragma unroll
    for (int c = 0; c < C; ++c)
        if (lane * C + c == E)
            out = P[c];
    return __shfl_sync(0xffffffffu, out, E / C);
}

}  // namespace ssk
