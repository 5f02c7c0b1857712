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
#include <type_traits>
#include <utility>

#include "ss_device.cuh"
#include "ss_rw_config.h"

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

// Any three-input bitwise function as one logic op: bit i of the result is
// bit (4 a_i + 2 b_i + c_i) of LUT.  Written as one lop3 so that the walk's
// steps stay one instruction each.  The tables used: 0x90 = a & ~(b ^ c),
// 0xFE = a | b | c, 0xF4 = a | (b & ~c), 0xF3 = a | ~b.
template <uint32_t LUT>
SS_HD uint32_t lop3(uint32_t a, uint32_t b, uint32_t c)
{
#ifdef __CUDA_ARCH__
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;"
        : "=r"(d)
        : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
#else
    uint32_t d = 0u;
    for (int k = 0; k < 8; ++k)
        if ((LUT >> k) & 1u)
            d |= ((k & 4) ? a : ~a) & ((k & 2) ? b : ~b) & ((k & 1) ? c : ~c);
    return d;
#endif
}

// OR of x[0..N-1] as a tree of three-input ORs (one logic op each).
template <int N>
SS_HD uint32_t or_tree(const uint32_t (&x)[N])
{
    if constexpr (N == 1) {
        return x[0];
    } else {
        constexpr int M = (N + 2) / 3;
        uint32_t y[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const uint32_t b = 3 * i + 1 < N ? x[3 * i + 1] : 0u;
            const uint32_t c = 3 * i + 2 < N ? x[3 * i + 2] : 0u;
            y[i] = 3 * i + 1 < N ? lop3<0xFE>(x[3 * i], b, c) : x[3 * i];
        }
        return or_tree<M>(y);
    }
}

// min(count, E+1) of the 32 pairs of a group, bit-sliced.  Below
// kSlicedBinaryFromE a thermometer: T[c] = pairs with count >= c, c = 1..E+1
// (E+1 logic ops per column, saturating by construction).  From it a
// saturating binary count: bit b of the count in c[b] (NB words) and the
// pairs that reached E+1 in dn; per column one op for the increment
// (restarted and not done), two per bit for the ripple and about NB/2 for
// "reached E+1" -- fewer registers than the thermometer, and fewer ops once
// E+1 passes about 12.  Measured at 30M x 100 bp: E = 7 0.364 ms with the
// thermometer against 0.367 binary; E = 8/9/10 0.392/0.447/0.486 against
// 0.384/0.432/0.463.
constexpr int kSlicedBinaryFromE = 8;

template <int E, bool BIN = (E >= kSlicedBinaryFromE)>
struct SlicedCount;

template <int E>
struct SlicedCount<E, false> {
    uint32_t T[E + 2];
    // pad: pairs that do not exist, counted as past E
    SS_HD void init(uint32_t pad)
    {
#pragma unroll
        for (int c = 0; c <= E; ++c)
            T[c] = 0u;
        T[E + 1] = pad;
    }
    // nz: the pairs with a row still alive at this column (the others
    // count one obstacle): T_c |= T_c-1 & ~nz, T_1 |= ~nz
    SS_HD void step(uint32_t nz)
    {
#pragma unroll
        for (int c = E + 1; c >= 2; --c)
            T[c] = lop3<0xF4>(T[c], T[c - 1], nz);
        T[1] = lop3<0xF3>(T[1], nz, 0u);
    }
    // pairs whose count reached E+1
    SS_HD uint32_t done() const { return T[E + 1]; }
    // binary bits of min(count, E+1): bit b is the XOR of T[c] over the
    // multiples c of 2^b (T[c] = count >= c, so that XOR is the parity of
    // floor(count / 2^b))
    SS_HD void bits(uint32_t (&cb)[SlicedShape<E>::NB]) const
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
};

template <int E>
struct SlicedCount<E, true> {
    static constexpr int NB = SlicedShape<E>::NB;
    uint32_t c[NB];
    uint32_t dn;  // pairs whose count is E+1 (and the padding)
    SS_HD void init(uint32_t pad)
    {
#pragma unroll
        for (int b = 0; b < NB; ++b)
            c[b] = 0u;
        dn = pad;
    }
    SS_HD void step(uint32_t nz)
    {
        // +1 for the pairs with every row dead, unless already at E+1
        uint32_t k = lop3<0x03>(nz, dn, 0u);  // ~(nz | dn)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const uint32_t x = c[b];
            c[b] = x ^ k;
            k &= x;
        }
        uint32_t eq = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            eq &= (((E + 1) >> b) & 1) ? c[b] : ~c[b];
        dn |= eq;
    }
    SS_HD uint32_t done() const { return dn; }
    SS_HD void bits(uint32_t (&cb)[NB]) const
    {
#pragma unroll
        for (int b = 0; b < NB; ++b)
            cb[b] = c[b];
    }
};

// The edge blocks of a walk over mR reference columns against a query of
// mQ bases (mQ = mR = m for pairs of equal length): a block k is an edge
// block when one of its columns has a diagonal that reads a query base
// outside 0..mQ-1 (Eq. 1 case 4): k < kl (j0 < E) or k >= kr (j0 + 3 + E >=
// mQ).  Their validity words -- all ones or zero per window word, the same
// for every pair -- are rows of a table: row k for k < kl, row kl +
// min(k, kz) - kr for k >= kr, where from block kz on the whole window lies
// past the query (every such block has the same row; only a reference
// longer than the query reaches it).  At most 2 NBH + 1 rows with equal
// lengths, 3 NBH + 2 otherwise.
template <int E>
struct SlicedEdges {
    static constexpr int kRows = 2 * SlicedShape<E>::NBH + 2;
    static constexpr int kRowsFree = 3 * SlicedShape<E>::NBH + 3;
    int nb, kl, kr, kz;
    SS_HD explicit SlicedEdges(int m) : SlicedEdges(m, m) {}
    SS_HD SlicedEdges(int mQ, int mR)
    {
        nb = (mR + 3) >> 2;
        kl = imin(nb, SlicedShape<E>::NBH);
        // first k with 4k + 3 + E >= mQ (at most nb: a query longer than
        // the reference may leave no right edge)
        const int r = mQ - 3 - E;
        kr = imin(nb, imax(kl, r <= 0 ? 0 : (r + 3) >> 2));
        // first k whose window (query bases 4k - 4 NBH ..) starts past the
        // query: at least nb with equal lengths
        kz = ((mQ + 3) >> 2) + SlicedShape<E>::NBH;
    }
    SS_HD int rows() const { return kl + (imin(nb, kz + 1) - kr); }
    SS_HD int row_of(int k) const
    {
        return k < kl ? k : kl + (imin(k, kz) - kr);
    }
    SS_HD int block_of(int row) const
    {
        return row < kl ? row : kr + (row - kl);
    }
    // validity word w of the window of block k (mQ: the query's bases)
    SS_HD static uint32_t valid(int k, int w, int mQ)
    {
        return (uint32_t)(4 * k - 4 * SlicedShape<E>::NBH + w) < (uint32_t)mQ
                   ? 0xffffffffu
                   : 0u;
    }
    // word w of block k's table row: with equal lengths the validity word
    // (a cell outside the query is an obstacle), with different lengths
    // its complement (such a cell is free: Section 2.4's correction)
    SS_HD static uint32_t entry(int k, int w, int mQ, bool free_ends)
    {
        const uint32_t v = valid(k, w, mQ);
        return free_ends ? ~v : v;
    }
};

// Column j0 + u of a block.  ql/qh: the window's query words (word w =
// query base j0 - 4 NBH + w); rl/rh: the reference bases j0..j0+3.  With
// EDGE, vw holds the block's table row: a diagonal that reads a query base
// outside 0..mQ-1 meets an obstacle (Eq. 1 case 4; vw the validity words)
// or, with FREE (the lengths differ), a free cell (vw their complement:
// S_d = (S_d | z) & (equal | outside)).  one holds 1 (a run-time value:
// S_d * one + z is a multiply-add on the FMA pipe).
// What a column adds to the greedy, by mode.  The plain walk: nothing.
struct SlicedPlain {
    template <int N>
    SS_HD void column_start(int, uint32_t (&)[N], uint32_t &)
    {
    }
    SS_HD uint32_t counted(uint32_t nz) const { return nz; }
    SS_HD void after(uint32_t) {}
};

// The sub-maze mode (Section 2.5): the maze cut into sub-mazes of t columns,
// each routed from its own first column (every row restarts there), with at
// most y escape segments counted per sub-maze (y taken as min(y, E+1): the
// count stops at E+1 anyway).  Per pair a binary count of the sub-maze's
// segments (NB words) and the pairs that reached y (frozen: their deaths
// are no longer counted in this sub-maze).
template <int E>
struct SlicedSubMaze {
    static constexpr int NB = SlicedShape<E>::NB;
    uint32_t sb[NB];
    uint32_t ym[NB];  // bit b of y, all ones or zero
    uint32_t frozen;
    int t, next;
    SS_HD SlicedSubMaze(int t_, int y)
    {
        t = t_;
        next = 0;
        const int ye = y < E + 1 ? y : E + 1;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            sb[b] = 0u;
            ym[b] = ((ye >> b) & 1) ? 0xffffffffu : 0u;
        }
        frozen = 0u;
    }
    // column j: a sub-maze's first column restarts every row of every pair
    // (S | z all ones; S cleared so that S | z stays S + z)
    template <int N>
    SS_HD void column_start(int j, uint32_t (&S)[N], uint32_t &z)
    {
        if (j == next) {
#pragma unroll
            for (int d = 0; d < N; ++d)
                S[d] = 0u;
            z = 0xffffffffu;
#pragma unroll
            for (int b = 0; b < NB; ++b)
                sb[b] = 0u;
            frozen = 0u;
            next += t;
        }
    }
    // frozen pairs count as alive (no obstacle counted)
    SS_HD uint32_t counted(uint32_t nz) const { return nz | frozen; }
    SS_HD void after(uint32_t nz)
    {
        uint32_t k = lop3<0x03>(nz, frozen, 0u);  // a counted death
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const uint32_t x = sb[b];
            sb[b] = x ^ k;
            k &= x;
        }
        uint32_t eq = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            eq = lop3<0x90>(eq, sb[b], ym[b]);  // eq & ~(sb ^ ym)
        frozen = eq;
    }
};

// The window may be wider than E needs (NW blocks either side, NW >= NBH):
// word w is then query base j0 - 4 NW + w.
template <int E, bool EDGE, int U, int NW = SlicedShape<E>::NBH,
          class Mode = SlicedPlain, bool FREE = false>
SS_HD void sliced_column(uint32_t (&S)[2 * E + 1], uint32_t &z,
                         SlicedCount<E> &cnt,
                         const uint32_t (&ql)[4 * (2 * NW + 1)],
                         const uint32_t (&qh)[4 * (2 * NW + 1)],
                         const uint32_t (&rl)[4], const uint32_t (&rh)[4],
                         const uint32_t *vw, uint32_t one, Mode &mode,
                         int j0)
{
    using Sh = SlicedShape<E>;
    static_assert(NW >= Sh::NBH, "window narrower than E needs");
    mode.column_start(j0 + U, S, z);
#pragma unroll
    for (int d = 0; d < Sh::ND; ++d) {
        const int w = 4 * NW - E + U + d;
        // (S_d | z) & ~(Q lo ^ R lo) & ~(Q hi ^ R hi)
        const uint32_t t = S[d] * one + z;
        uint32_t s = lop3<0x90>(t, ql[w], rl[U]);
        s = lop3<0x90>(s, qh[w], rh[U]);
        if (EDGE)
            s = FREE ? lop3<0xF8>(s, t, vw[w]) : (s & vw[w]);  // s | (t & vw)
        S[d] = s;
    }
    // the pairs with every row dead: count this column's obstacle,
    // restart at the next column
    const uint32_t nz = or_tree<Sh::ND>(S);
    cnt.step(mode.counted(nz));
    mode.after(nz);
    z = ~nz;
}

// The block's columns j0 + u for u < live (1..4; below 4 only in the last
// block).
template <int E, bool EDGE, class Mode, bool FREE = false>
SS_HD void sliced_block(uint32_t (&S)[2 * E + 1], uint32_t &z,
                        SlicedCount<E> &cnt,
                        const uint32_t (&ql)[SlicedShape<E>::WW],
                        const uint32_t (&qh)[SlicedShape<E>::WW],
                        const uint32_t (&rl)[4], const uint32_t (&rh)[4],
                        const uint32_t *vw, int live, uint32_t one,
                        Mode &mode, int j0)
{
    constexpr int NW = SlicedShape<E>::NBH;
    auto col = [&](auto u) {
        sliced_column<E, EDGE, decltype(u)::value, NW, Mode, FREE>(
            S, z, cnt, ql, qh, rl, rh, vw, one, mode, j0);
    };
    using std::integral_constant;
    if (live >= 4) {
        col(integral_constant<int, 0>{});
        col(integral_constant<int, 1>{});
        col(integral_constant<int, 2>{});
        col(integral_constant<int, 3>{});
    } else {
        col(integral_constant<int, 0>{});
        if (live > 1)
            col(integral_constant<int, 1>{});
        if (live > 2)
            col(integral_constant<int, 2>{});
    }
}

// Walk the 32 pairs of one group over all mR reference columns against
// queries of mQ bases (FREE: mQ != mR, Section 2.4's correction; else mQ =
// mR); on return cnt holds each pair's min(count, E+1).  pad: pairs that
// do not exist (the last group's), counted as past E so that the group can
// stop early.  src.query(blk, nb, lo, hi) / src.ref(blk, lo, hi) load the
// four words of each plane of a block (zero for a query block outside
// 0..nb-1); src.prefetch(qblk, rblk, nbq, nbr) asks for those of query
// block qblk (if below nbq) and reference block rblk (if below nbr) ahead
// of their loads (a hint, no result);
// vtab: the table of SlicedEdges<E>(mQ, mR), WW words per row (entry()).
template <int E, bool FREE, class Src, class Mode = SlicedPlain>
SS_HD void sliced_walk2(const Src &src, int mQ, int mR, uint32_t pad,
                        SlicedCount<E> &cnt, const uint32_t *vtab,
                        uint32_t one, Mode mode = Mode())
{
    using Sh = SlicedShape<E>;
    const SlicedEdges<E> ed(mQ, mR);
    const int nb = ed.nb;                       // reference blocks
    const int nbq = FREE ? (mQ + 3) >> 2 : nb;  // query blocks
    const int m = mR;
    uint32_t ql[Sh::WW], qh[Sh::WW];
#pragma unroll
    for (int b = 0; b < 2 * Sh::NBH + 1; ++b) {
        uint32_t lo[4], hi[4];
        src.query(b - Sh::NBH, nbq, lo, hi);
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
    cnt.init(pad);
    uint32_t rl[4], rh[4];
    if (nb > 0)
        src.ref(0, rl, rh);
    // where the rows and the window fill the registers, the next block's
    // words are prefetched to L1 instead of held, and loaded into the
    // window after it slides: from E = 25 (10M x 250 bp: E = 24 0.82 ms
    // held against 0.87 prefetched, E = 25 1.00 held, with spills, against
    // 0.86), and at E = 10-11, where it brings the kernel to 128 registers
    // (4 CTAs per SM; 30M x 100 bp E = 10 0.463 -> 0.457 ms; slower at
    // E = 7 and 12-15)
    constexpr bool kHold = E < 10 || (E > 11 && E < 25);
    for (int k = 0; k < nb; ++k) {
        uint32_t nql[4], nqh[4], nrl[4], nrh[4];
        if constexpr (kHold) {
            // the next block's words, loaded before this block is walked
            src.query(k + Sh::NBH + 1, nbq, nql, nqh);
            if (k + 1 < nb)
                src.ref(k + 1, nrl, nrh);
        } else {
            src.prefetch(k + Sh::NBH + 1, k + 1, nbq, nb);
        }
        const int live = imin(4, m - 4 * k);
        if (k < ed.kl || k >= ed.kr)
            sliced_block<E, true, Mode, FREE>(S, z, cnt, ql, qh, rl, rh,
                                              vtab + ed.row_of(k) * Sh::WW,
                                              live, one, mode, 4 * k);
        else
            sliced_block<E, false, Mode, FREE>(S, z, cnt, ql, qh, rl, rh,
                                               nullptr, live, one, mode,
                                               4 * k);
        if (cnt.done() == 0xffffffffu)
            break;  // every pair of the group is past E
#pragma unroll
        for (int w = 0; w + 4 < Sh::WW; ++w) {
            ql[w] = ql[w + 4];
            qh[w] = qh[w + 4];
        }
        if constexpr (!kHold) {
            src.query(k + Sh::NBH + 1, nbq, nql, nqh);
            if (k + 1 < nb)
                src.ref(k + 1, nrl, nrh);
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

// The walk of pairs of equal length m.
template <int E, class Src, class Mode = SlicedPlain>
SS_HD void sliced_walk(const Src &src, int m, uint32_t pad,
                       SlicedCount<E> &cnt, const uint32_t *vtab,
                       uint32_t one, Mode mode = Mode())
{
    sliced_walk2<E, false>(src, m, m, pad, cnt, vtab, one, mode);
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
    // whole bytes and half-words: one byte permute of the two words
    if (d == 16)
        return prmt(v, x, keep_low ? 0x5410u : 0x3276u);
    if (d == 8)
        return prmt(v, x, keep_low ? 0x6240u : 0x3715u);
    uint32_t ml;  // bits whose index has bit d clear
    switch (d) {
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

namespace ssk {

// ---- several thresholds in one pass over the data ------------------------
// Thresholds whose walks cost less than streaming the pairs (E <= 4 at
// 100 bp) share one pass: one query window (sized for the largest E), one
// set of reference words and one edge table, and per threshold its own
// rows, restart word and count.  Each threshold's walk is exactly the
// single-threshold walk above; only the loads are shared.


// One threshold's state.
template <int E>
struct SlicedTrack {
    uint32_t S[2 * E + 1];
    uint32_t z;
    SlicedCount<E> cnt;
    SS_HD void init(uint32_t pad)
    {
#pragma unroll
        for (int d = 0; d < 2 * E + 1; ++d)
            S[d] = 0xffffffffu;
        z = 0u;
        cnt.init(pad);
    }
};

template <int... Es>
struct SlicedTracks;

template <>
struct SlicedTracks<> {
    SS_HD void init(uint32_t) {}
    SS_HD uint32_t done() const { return 0xffffffffu; }
};

template <int E, int... R>
struct SlicedTracks<E, R...> {
    SlicedTrack<E> head;
    SlicedTracks<R...> tail;
    SS_HD void init(uint32_t pad)
    {
        head.init(pad);
        tail.init(pad);
    }
    // pairs past E for every threshold of the set
    SS_HD uint32_t done() const { return head.cnt.done() & tail.done(); }
};

// Column U of a block for every threshold of the set (window of NW blocks
// either side).
template <int NW, bool EDGE, int U>
SS_HD void set_column(SlicedTracks<> &, const uint32_t (&)[4 * (2 * NW + 1)],
                      const uint32_t (&)[4 * (2 * NW + 1)],
                      const uint32_t (&)[4], const uint32_t (&)[4],
                      const uint32_t *, uint32_t)
{
}

template <int NW, bool EDGE, int U, int E, int... R>
SS_HD void set_column(SlicedTracks<E, R...> &t,
                      const uint32_t (&ql)[4 * (2 * NW + 1)],
                      const uint32_t (&qh)[4 * (2 * NW + 1)],
                      const uint32_t (&rl)[4], const uint32_t (&rh)[4],
                      const uint32_t *vw, uint32_t one)
{
    SlicedPlain plain;
    sliced_column<E, EDGE, U, NW>(t.head.S, t.head.z, t.head.cnt, ql, qh, rl,
                                  rh, vw, one, plain, 0);
    set_column<NW, EDGE, U>(t.tail, ql, qh, rl, rh, vw, one);
}

template <int NW, bool EDGE, int... Es>
SS_HD void set_block(SlicedTracks<Es...> &t,
                     const uint32_t (&ql)[4 * (2 * NW + 1)],
                     const uint32_t (&qh)[4 * (2 * NW + 1)],
                     const uint32_t (&rl)[4], const uint32_t (&rh)[4],
                     const uint32_t *vw, int live, uint32_t one)
{
    set_column<NW, EDGE, 0>(t, ql, qh, rl, rh, vw, one);
    if (live > 1)
        set_column<NW, EDGE, 1>(t, ql, qh, rl, rh, vw, one);
    if (live > 2)
        set_column<NW, EDGE, 2>(t, ql, qh, rl, rh, vw, one);
    if (live > 3)
        set_column<NW, EDGE, 3>(t, ql, qh, rl, rh, vw, one);
}

// The walk of sliced_walk for every threshold of the ascending set Es
// (largest EMAX) over one group; vtab: the validity table of
// SlicedEdges<EMAX>(m).
template <int EMAX, class Src, int... Es>
SS_HD void sliced_walk_set(const Src &src, int m, uint32_t pad,
                           SlicedTracks<Es...> &t, const uint32_t *vtab,
                           uint32_t one)
{
    constexpr int NW = SlicedShape<EMAX>::NBH;
    constexpr int WW = SlicedShape<EMAX>::WW;
    const SlicedEdges<EMAX> ed(m);
    const int nb = ed.nb;
    uint32_t ql[WW], qh[WW];
#pragma unroll
    for (int b = 0; b < 2 * NW + 1; ++b) {
        uint32_t lo[4], hi[4];
        src.query(b - NW, nb, lo, hi);
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            ql[4 * b + x] = lo[x];
            qh[4 * b + x] = hi[x];
        }
    }
    t.init(pad);
    uint32_t rl[4], rh[4];
    if (nb > 0)
        src.ref(0, rl, rh);
    for (int k = 0; k < nb; ++k) {
        uint32_t nql[4], nqh[4], nrl[4], nrh[4];
        src.query(k + NW + 1, nb, nql, nqh);
        if (k + 1 < nb)
            src.ref(k + 1, nrl, nrh);
        const int live = imin(4, m - 4 * k);
        if (k < ed.kl || k >= ed.kr)
            set_block<NW, true>(t, ql, qh, rl, rh,
                                vtab + ed.row_of(k) * WW, live, one);
        else
            set_block<NW, false>(t, ql, qh, rl, rh, nullptr, live, one);
        if (t.done() == 0xffffffffu)
            break;  // every pair past every threshold
#pragma unroll
        for (int w = 0; w + 4 < WW; ++w) {
            ql[w] = ql[w + 4];
            qh[w] = qh[w + 4];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            ql[WW - 4 + x] = nql[x];
            qh[WW - 4 + x] = nqh[x];
            rl[x] = nrl[x];
            rh[x] = nrh[x];
        }
    }
}

// The thresholds of a bit mask (bit e: threshold e), ascending.
template <unsigned MASK, int B, int... Es>
struct MaskThresholds {
    using type = typename std::conditional<
        ((MASK >> B) & 1u) != 0u,
        typename MaskThresholds<MASK, B + 1, Es..., B>::type,
        typename MaskThresholds<MASK, B + 1, Es...>::type>::type;
};
template <unsigned MASK, int... Es>
struct MaskThresholds<MASK, kSlicedSetMaxE + 1, Es...> {
    using type = std::integer_sequence<int, Es...>;
};

}  // namespace ssk

#ifdef __CUDACC__
namespace ssk {

// ---- device side: one group's words in global memory, results -----------

constexpr int kSlicedThreads = 128;

// Reads or refs in the layout: uint4 index (blk * G + g) * 2 + b.
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
    __device__ __forceinline__ void prefetch(int qblk, int rblk, int nbq,
                                             int nbr) const
    {
        if (qblk >= 0 && qblk < nbq)
            asm volatile("prefetch.global.L1 [%0];"
                         :
                         : "l"(q + ((int64_t)qblk * G + g) * 2));
        if (rblk < nbr)
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

// The validity table of the edge blocks, the same for every thread of the
// CTA (all threads call this, then synchronise).
template <int E>
__device__ __forceinline__ void sliced_fill_edges(uint32_t *vtab, int m)
{
    using Ed = SlicedEdges<E>;
    constexpr int WW = SlicedShape<E>::WW;
    const Ed ed(m);
    for (int i = threadIdx.x; i < ed.rows() * WW; i += kSlicedThreads)
        vtab[i] = Ed::valid(ed.block_of(i / WW), i % WW, m);
}

// The table of a walk over mR reference columns against queries of mQ
// bases, with the free-end rule when they differ (SlicedEdges::entry).
template <int E>
__device__ __forceinline__ void sliced_fill_edges2(uint32_t *vtab, int mQ,
                                                   int mR)
{
    using Ed = SlicedEdges<E>;
    constexpr int WW = SlicedShape<E>::WW;
    const Ed ed(mQ, mR);
    for (int i = threadIdx.x; i < ed.rows() * WW; i += kSlicedThreads)
        vtab[i] = Ed::entry(ed.block_of(i / WW), i % WW, mQ, mQ != mR);
}

// Results of the group's np pairs starting at pair p0: accept (count <= E,
// Section 2.4 step 5) and min(count, E+1); vec: acc and obs 16-byte
// aligned, so a whole group is stored with 16-byte stores.
template <int E>
__device__ __forceinline__ void sliced_store(const SlicedCount<E> &cnt,
                                             uint8_t *acc, int32_t *obs,
                                             int64_t p0, int np, bool vec)
{
    uint32_t cb[SlicedShape<E>::NB];
    cnt.bits(cb);
    const uint32_t ok = ~cnt.done();
    if (np == 32 && vec) {
        uint4 *o = reinterpret_cast<uint4 *>(obs + p0);
#pragma unroll
        for (int v = 0; v < 8; ++v)
            o[v] = make_uint4((uint32_t)sliced_count<E>(cb, 4 * v),
                              (uint32_t)sliced_count<E>(cb, 4 * v + 1),
                              (uint32_t)sliced_count<E>(cb, 4 * v + 2),
                              (uint32_t)sliced_count<E>(cb, 4 * v + 3));
        uint4 *f = reinterpret_cast<uint4 *>(acc + p0);
        f[0] = make_uint4(flag_bytes(ok, 0), flag_bytes(ok, 1),
                          flag_bytes(ok, 2), flag_bytes(ok, 3));
        f[1] = make_uint4(flag_bytes(ok, 4), flag_bytes(ok, 5),
                          flag_bytes(ok, 6), flag_bytes(ok, 7));
    } else {
        for (int i = 0; i < np; ++i) {
            obs[p0 + i] = sliced_count<E>(cb, i);
            acc[p0 + i] = (uint8_t)((ok >> i) & 1u);
        }
    }
}

}  // namespace ssk
#endif
