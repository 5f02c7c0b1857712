// ss_sliced.cuh -- the bit-sliced layout (SS_FMT_SLICED2) and the filter
// over it: one thread walks the mazes of 32 pairs at once, one pair per bit.
//
// Layout (include/ss.h): pairs in groups of 32, pair p = bit p%32 of group
// g = p/32 (G groups); code bit b of base j of the group's 32 sequences is
// one word, at index ((j/4 * G + g) * 2 + b) * 4 + j%4.  A thread's four
// consecutive bases of one code bit are one 16-byte load, and the 32
// threads of a warp (32 consecutive groups) read 1 KB contiguous per block
// of four bases.  100 bases take 25 bytes per sequence, 2 bits per base.
//
// Method (Section 2.4, walked one column at a time): from a checkpoint c
// the longest escape segment ends where the last maze row free of
// obstacles since c meets its obstacle.  With S_d = the pairs whose row d
// (diagonal s = d - E) is free since their checkpoint, one column j is, for
// every d,
//     S_d = (S_d | z) & [Q[j + s] == R[j]]          (Eq. 1; case 4 below)
// where z = the pairs all of whose rows died at column j-1 (each such pair
// counts that obstacle and restarts at column j with every row free), and
// the column's own z is the pairs with every S_d now empty.  A pair that
// reaches column m-1 with a row alive ends with no further count.  The
// count is kept as a thermometer, T_c = pairs with count >= c for c = 1..
// E+1, so it saturates at E+1 (Section 2.4 step 4 stops there).
//
// Cost per column and 32 pairs: two three-input logic ops per diagonal (the
// equality of the two code bits), one add per diagonal (S_d | z is S_d + z,
// since z's pairs have every S_d empty; the add issues on the FMA pipe), E
// three-input ORs for the column's z and E+1 ops of the thermometer: 6E+3
// logic ops and 2E+1 adds for 32 pairs, where one pair per thread costs
// about eight ops per column.  There is no early exit per pair (a group
// stops when all of its 32 pairs are past E), and no cost order: the work
// of a group does not depend on how similar its pairs are.
#pragma once
#include <cstdint>

#include "ss_device.cuh"

namespace ssk {

// Shape of the walk at threshold E: a block of four columns reads query
// bases up to E before its first and after its last column, so the query
// window holds NBH blocks either side of the current one.
template <int E>
struct SlicedShape {
    static constexpr int ND = 2 * E + 1;          // maze rows (diagonals)
    static constexpr int NBH = (E + 3) / 4;       // window blocks per side
    static constexpr int WW = 4 * (2 * NBH + 1);  // window words per plane
    // window word of the query base that diagonal 0 (s = -E) reads at the
    // block's first column: the window starts 4 NBH bases before it
    static constexpr int OFF = 4 * NBH - E;
    // bits of E+1 (the largest count kept)
    static constexpr int NB = E + 1 >= 32 ? 6
                              : E + 1 >= 16 ? 5
                              : E + 1 >= 8  ? 4
                              : E + 1 >= 4  ? 3
                              : E + 1 >= 2  ? 2
                                            : 1;
};

// The block's columns j0 + u for u < live (at most 4).  ql/qh: the window's
// query words (word w = query base j0 - 4 NBH + w); rl/rh: the reference
// bases j0..j0+3.  With EDGE, a diagonal that reads a query base outside
// 0..m-1 meets an obstacle (Eq. 1 case 4); without, every base read is in
// range.  one holds 1 (a run-time value: S_d * one + z is a multiply-add).
template <int E, bool EDGE>
SS_HD void sliced_block(uint32_t (&S)[2 * E + 1], uint32_t &z,
                        uint32_t (&T)[E + 2],
                        const uint32_t (&ql)[SlicedShape<E>::WW],
                        const uint32_t (&qh)[SlicedShape<E>::WW],
                        const uint32_t (&rl)[4], const uint32_t (&rh)[4],
                        int j0, int m, int live, uint32_t one)
{
    using Sh = SlicedShape<E>;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (u < live) {
            uint32_t nz = 0u;
#pragma unroll
            for (int d = 0; d < Sh::ND; ++d) {
                const int w = Sh::OFF + u + d;
                uint32_t s = S[d] * one + z;
                s &= ~(ql[w] ^ rl[u]);
                s &= ~(qh[w] ^ rh[u]);
                if (EDGE) {
                    const int qi = j0 + u + d - E;
                    if (qi < 0 || qi >= m)
                        s = 0u;
                }
                S[d] = s;
                nz |= s;
            }
            z = ~nz;
#pragma unroll
            for (int c = E + 1; c >= 2; --c)
                T[c] |= T[c - 1] & z;
            T[1] |= z;
        }
    }
}

// Walk the 32 pairs of one group over all m columns; on return T[c] (c =
// 1..E+1) holds the pairs whose count reached c, i.e. bit i of the pair's
// min(count, E+1) in thermometer form.  pad: pairs that do not exist (the
// last group's), counted as past E so that the group can stop early.
// src.query(blk, nb, lo, hi) / src.ref(blk, lo, hi) load the four words of
// each plane of a block (zero for a query block outside 0..nb-1).
template <int E, class Src>
SS_HD void sliced_walk(const Src &src, int m, uint32_t pad,
                       uint32_t (&T)[E + 2], uint32_t one)
{
    using Sh = SlicedShape<E>;
    const int nb = (m + 3) >> 2;
    uint32_t ql[Sh::WW], qh[Sh::WW];
#pragma unroll
    for (int b = 0; b < 2 * Sh::NBH + 1; ++b) {
        uint32_t lo[4], hi[4];
        src.query(b - Sh::NBH, nb, lo, hi);
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            ql[4 * b + x] = lo[x];
            qh[4 * b + x] = hi[x];
        }
    }
    uint32_t S[Sh::ND];
#pragma unroll
    for (int d = 0; d < Sh::ND; ++d)
        S[d] = 0xffffffffu;
    uint32_t z = 0u;
#pragma unroll
    for (int c = 0; c <= E; ++c)
        T[c] = 0u;
    T[E + 1] = pad;
    uint32_t rl[4], rh[4];
    if (nb > 0)
        src.ref(0, rl, rh);
    for (int k = 0; k < nb; ++k) {
        // the next block's words, loaded before this block is walked
        uint32_t nql[4], nqh[4], nrl[4], nrh[4];
        src.query(k + Sh::NBH + 1, nb, nql, nqh);
        if (k + 1 < nb)
            src.ref(k + 1, nrl, nrh);
        const int j0 = 4 * k;
        const int live = imin(4, m - j0);
        if (j0 < E || j0 + 3 + E >= m)
            sliced_block<E, true>(S, z, T, ql, qh, rl, rh, j0, m, live, one);
        else
            sliced_block<E, false>(S, z, T, ql, qh, rl, rh, j0, m, live, one);
        if (T[E + 1] == 0xffffffffu)
            break;  // every pair of the group is past E
#pragma unroll
        for (int w = 0; w + 4 < Sh::WW; ++w) {
            ql[w] = ql[w + 4];
            qh[w] = qh[w + 4];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            ql[Sh::WW - 4 + x] = nql[x];
            qh[Sh::WW - 4 + x] = nqh[x];
            rl[x] = nrl[x];
            rh[x] = nrh[x];
        }
    }
}

// Binary bits of the thermometer count: bit b of min(count, E+1) is the XOR
// of T[c] over the multiples c of 2^b (T[c] = count >= c, so that XOR is
// the parity of floor(count / 2^b)).
template <int E>
SS_HD void sliced_binary(const uint32_t (&T)[E + 2],
                         uint32_t (&cb)[SlicedShape<E>::NB])
{
#pragma unroll
    for (int b = 0; b < SlicedShape<E>::NB; ++b) {
        uint32_t x = 0u;
#pragma unroll
        for (int c = 1 << b; c <= E + 1; c += 1 << b)
            x ^= T[c];
        cb[b] = x;
    }
}

// min(count, E+1) of pair i of the group.
template <int E>
SS_HD int sliced_count(const uint32_t (&cb)[SlicedShape<E>::NB], int i)
{
    int c = 0;
#pragma unroll
    for (int b = 0; b < SlicedShape<E>::NB; ++b)
        c |= (int)((cb[b] >> i) & 1u) << b;
    return c;
}

// One level of the 32 x 32 bit transpose across a warp (lanes x bits): lane
// `lane` holds v, its partner lane ^ d holds x.  A lane with bit d of its
// index clear keeps its bits whose index has bit d clear and takes the
// partner's such bits into the positions with bit d set; the other lane
// the converse.  After the levels d = 16, 8, 4, 2, 1, lane r holds bit r
// of every lane's word (bit i from lane i).
SS_HD uint32_t transpose_level(uint32_t v, uint32_t x, int lane, int d)
{
    const bool keep_low = (lane & d) == 0;
    uint32_t ml;  // bits whose index has bit d clear
    switch (d) {
    case 16: ml = 0x0000ffffu; break;
    case 8: ml = 0x00ff00ffu; break;
    case 4: ml = 0x0f0f0f0fu; break;
    case 2: ml = 0x33333333u; break;
    default: ml = 0x55555555u; break;
    }
    // the partner's bits, moved by d: up (rotate left) for the low lane,
    // down (rotate right) for the other
    const uint32_t y = funnel_l(x, x, keep_low ? (uint32_t)d : 32u - d);
    const uint32_t k = keep_low ? ml : ~ml;
    return (v & k) | (y & ~k);
}

}  // namespace ssk
