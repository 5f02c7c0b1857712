// ss_rwc.cuh -- one thread per pair, the greedy walked one column at a time
// with the 2E+1 maze rows as the bits of one word (E <= 15) or two (E =
// 16..31).
//
// Method (Section 2.4): from checkpoint c the longest escape segment ends
// at p* = max over rows of the row's first obstacle at or after c.  Walking
// the columns j = c, c+1, ... with S_j = the rows free of obstacles in
// columns c..j (S_c-1 = all rows), p* is the first j with S_j = 0: the
// column where the last surviving row meets its obstacle.  That obstacle is
// counted and the walk restarts at p* + 1 with all rows; reaching the row
// end with S non-empty ends the net with no count.  The walk stops once the
// count exceeds E (only min(count, E+1) is reported).
//
// GB300 mapping: the surviving rows are the bits of one word (2E+1 <= 32)
// or two.  Column j of the maze (Eq. 1) is compared in one logic op per
// bit plane and word: the Q planes around j against R[j] broadcast to
// every row (a byte permute of a multiply-spread R word), ANDed into the
// survivors -- and, only in chunks where a row can leave the query, the
// "Q base exists" plane (Eq. 1 case 4).  Two forms:
//  * frame form (most E): for a chunk of 8 (or 4) columns the Q planes are
//    one fixed frame of one or two words, and the survivors move one bit
//    up per column (a multiply by two on the FMA pipe);
//  * Q-shift form (E = 15, 31): the survivors keep their bits and each
//    column takes its Q windows with one funnel shift per plane and word.
// About eight integer operations per column with one survivor word (the
// frame form), and every thread of a warp executes the same column body,
// so a warp diverges only where its pairs stop.  Cheaper than the row-wise routing (rw_route) once 2E+1 rows
// are many and many pairs are dissimilar: a random pair is rejected after
// a few columns per obstacle, where row-wise routing rebuilds and scans all
// rows of each word (for a long, similar pair the row-wise form, 32
// columns per op, stays cheaper).  The same walk, with the pair's rows
// masked inside a wider word, serves the sub-maze mode (ss_submaze.cuh) and
// pairs of different lengths (ss_unequal.cuh).
#pragma once
#include <cstdint>
#include <utility>

#include "ss_device.cuh"

namespace ssk {

// Bits 0..3 of r moved to the sign bits of the four bytes (bit i to bit
// 8i + 7).  The product's terms, bit i times 2^(7 + 7k) for k = 0..3, land
// on sixteen distinct positions, so nothing carries.
SS_HD uint32_t spread4(uint32_t r) { return (r & 0xfu) * 0x10204080u; }

// All ones if the sign bit of byte I of t is set, else zero: the byte
// permute's sign-replicating selector (selector nibble 8 + I), as an
// immediate operand.  Only bytes of the first source are selected, so t
// also serves as the second.
template <int I>
SS_HD uint32_t byte_sign(uint32_t t)
{
    static_assert(I >= 0 && I < 4, "byte index");
#ifdef __CUDA_ARCH__
    uint32_t d;
    asm("prmt.b32 %0, %1, %1, %2;"
        : "=r"(d)
        : "r"(t), "n"(0x8888 + 0x1111 * I));
    return d;
#else
    return ((t >> (8 * I + 7)) & 1u) ? 0xffffffffu : 0u;
#endif
}

// 32 bits of a plane from bit O of word C on (-32 < O < 32): the previous
// word P supplies negative offsets, the next word N positive ones.
template <int O>
SS_HD uint32_t rwc_window(uint32_t P, uint32_t C, uint32_t N)
{
    if constexpr (O < 0)
        return funnel_r(P, C, 32 + O);
    else
        return funnel_r(C, N, O);
}

// The Q planes around the 32-column word being walked: previous, current
// and next words of the lo, hi and "base exists" planes.
struct RwcQ {
    uint32_t lo_p, lo_c, lo_n, hi_p, hi_c, hi_n, v_p, v_c, v_n;
};

// 32 bits of a plane from bit O of word C on, 1 <= O < 64, for the upper
// word of a two-word frame: no row reads past word N (the highest Q index
// a chunk reads is its last column plus E <= 31), so the bits shifted in
// above N are never looked at.
template <int O>
SS_HD uint32_t rwc_window_up(uint32_t C, uint32_t N)
{
    static_assert(O >= 1 && O < 64, "offset");
    if constexpr (O < 32)
        return funnel_r(C, N, O);
    else
        return N >> (O - 32);
}

// ---- Q-shift form: the survivors keep their bit, the Q planes move ------
// Each column takes its Q windows with one funnel shift per plane and
// survivor word.  Used where the frame form's chunk would shrink to two
// columns (E = 15 and E = 31), whose per-chunk set-up costs more than the
// shifts it saves.

// The rows still free of obstacles since the checkpoint (bit i = diagonal
// s = i - E).  With 2E+1 <= 32 rows one word holds them; with 33..63 rows
// (E = 16..31) s0 holds rows 0..31 and s1 rows 32..2E.
template <int E>
struct RwcSurv {
    static constexpr bool kWide = 2 * E + 1 > 32;
    static constexpr uint32_t kAll0 =
        kWide ? 0xffffffffu : (uint32_t)((1ull << (2 * E + 1)) - 1u);
    static constexpr uint32_t kAll1 =
        kWide ? (uint32_t)((1ull << (2 * E + 1 - 32)) - 1u) : 0u;
    uint32_t s0 = kAll0, s1 = kAll1;
};

// Column D of the word (before the row end); tl/th: the R bits of D's
// quad of columns, spread by spread4.
template <int E, bool EDGE, int D>
SS_HD void rwq_column(RwcSurv<E> &S, int &count, const RwcQ &q, uint32_t tl,
                      uint32_t th)
{
    constexpr int O = D - E;  // Q bit of row 0 relative to the word
    const uint32_t bl = byte_sign<D & 3>(tl);
    const uint32_t bh = byte_sign<D & 3>(th);
    // one three-input logic op per plane: S & ~(Q plane ^ broadcast R bit)
    S.s0 &= ~(rwc_window<O>(q.lo_p, q.lo_c, q.lo_n) ^ bl);
    S.s0 &= ~(rwc_window<O>(q.hi_p, q.hi_c, q.hi_n) ^ bh);
    if (EDGE)
        S.s0 &= rwc_window<O>(q.v_p, q.v_c, q.v_n);
    bool z;
    if constexpr (RwcSurv<E>::kWide) {
        // rows 32..2E: Q bits from O + 32 on (O + 32 >= 1 since E <= 31)
        S.s1 &= ~(rwc_window_up<O + 32>(q.lo_c, q.lo_n) ^ bl);
        S.s1 &= ~(rwc_window_up<O + 32>(q.hi_c, q.hi_n) ^ bh);
        if (EDGE)
            S.s1 &= rwc_window_up<O + 32>(q.v_c, q.v_n);
        z = (S.s0 | S.s1) == 0u;
        S.s1 = z ? RwcSurv<E>::kAll1 : S.s1;
    } else {
        z = S.s0 == 0u;
    }
    // the last surviving row met its obstacle here: count it, restart
    count += z;
    S.s0 = z ? RwcSurv<E>::kAll0 : S.s0;
}

// Columns D0+I of the word for I in the sequence; with TAIL, only those
// with I < live (the row end's partial chunk: a uniform test per column).
template <int E, bool EDGE, int D0, bool TAIL, int... I>
SS_HD void rwq_columns(RwcSurv<E> &S, int &count, const RwcQ &q, uint32_t l0,
                       uint32_t h0, uint32_t l1, uint32_t h1, int live,
                       std::integer_sequence<int, I...>)
{
    ((!TAIL || I < live
          ? rwq_column<E, EDGE, D0 + I>(S, count, q, I < 4 ? l0 : l1,
                                        I < 4 ? h0 : h1)
          : void()),
     ...);
}

// Columns D0 .. D0+7 of the word (the first `live` of them with TAIL).
template <int E, bool EDGE, int D0, bool TAIL = false>
SS_HD void rwq_chunk(RwcSurv<E> &S, int &count, const RwcQ &q, uint32_t rlo,
                     uint32_t rhi, int live = 8)
{
    const uint32_t l0 = spread4(rlo >> D0), h0 = spread4(rhi >> D0);
    const uint32_t l1 = spread4(rlo >> (D0 + 4));
    const uint32_t h1 = spread4(rhi >> (D0 + 4));
    rwq_columns<E, EDGE, D0, TAIL>(S, count, q, l0, h0, l1, h1, live,
                                   std::make_integer_sequence<int, 8>{});
}

// Chunk D0 of the word at column base: the walk's result if it ends here
// (the row end, or the count past E), else -1.  A chunk is an edge chunk
// when one of its rows reads a query index below 0 or at/after m.
template <int E, int D0>
SS_HD int rwq_chunk_at(RwcSurv<E> &S, int &count, const RwcQ &q, uint32_t rlo,
                       uint32_t rhi, int base, int m)
{
    const int c0 = base + D0;
    if (c0 + 8 > m) {
        rwq_chunk<E, true, D0, true>(S, count, q, rlo, rhi, m - c0);
        return count <= E ? count : E + 1;
    }
    if (c0 < E || c0 + 7 + E >= m)
        rwq_chunk<E, true, D0>(S, count, q, rlo, rhi);
    else
        rwq_chunk<E, false, D0>(S, count, q, rlo, rhi);
    return count > E ? E + 1 : -1;
}

// Route one pair of length m with threshold E (1 <= E <= 31); returns
// min(count, E+1), equal to rw_route's.  Reads the Q words up to the one
// after the word being walked (planes k+1), as rw_route does.
template <int E, class Seq>
SS_HD int rw_route_qshift(const Seq &Qs, const Seq &Rs, int m)
{
    static_assert(E >= 1 && E <= 31, "2E+1 rows in at most two words");
    const int W32 = (m + 31) >> 5;
    RwcQ q;
    q.lo_p = q.hi_p = q.v_p = 0u;  // before the query: case 4
    Qs.planes(0, q.lo_c, q.hi_c);
    Qs.planes(1, q.lo_n, q.hi_n);
    q.v_c = mask_below(m);
    q.v_n = mask_below(m - 32);
    RwcSurv<E> S;
    int count = 0;
    for (int k = 0; k < W32; ++k) {
        const int base = k << 5;
        uint32_t rlo, rhi;
        Rs.planes(k, rlo, rhi);
        int res;
        if ((res = rwq_chunk_at<E, 0>(S, count, q, rlo, rhi, base, m)) >= 0 ||
            (res = rwq_chunk_at<E, 8>(S, count, q, rlo, rhi, base, m)) >= 0 ||
            (res = rwq_chunk_at<E, 16>(S, count, q, rlo, rhi, base, m)) >= 0 ||
            (res = rwq_chunk_at<E, 24>(S, count, q, rlo, rhi, base, m)) >= 0)
            return res;
        // slide the Q windows by one word
        q.lo_p = q.lo_c;
        q.hi_p = q.hi_c;
        q.v_p = q.v_c;
        q.lo_c = q.lo_n;
        q.hi_c = q.hi_n;
        q.v_c = q.v_n;
        Qs.planes(k + 2, q.lo_n, q.hi_n);
        q.v_n = mask_below(m - 32 * (k + 2));
    }
    return count <= E ? count : E + 1;
}

// ---- frame form: the Q planes stay put for a chunk, the survivors move ---

// Shape of the walk for threshold E.  The columns are walked in chunks of
// KC; within a chunk the Q planes stay put in a frame of W words whose
// bit b is Q index c0 - E + b (c0: the chunk's first column), and the
// surviving rows are kept in frame coordinates: at column c0 + d, row s
// (diagonal s = -E..E) is bit d + s + E.  Moving one column right moves
// every row one bit up, a multiply by two, where the other form shifts
// both Q planes (two funnel shifts on the ALU pipe).  Rows reach bit
// KC - 1 + 2E, so KC is the widest of 8, 4, 2 with 2E + KC <= 32 W.
template <int E>
struct RwcFrame {
    static_assert(E >= 1 && E <= 31, "2E+1 rows in at most two words");
    static constexpr int W = 2 * E + 1 > 32 ? 2 : 1;
    static constexpr int KC = 2 * E + 8 <= 32 * W   ? 8
                              : 2 * E + 4 <= 32 * W ? 4
                                                    : 2;
    static constexpr uint64_t kAll = (1ull << (2 * E + 1)) - 1ull;
    // every row alive, placed as at column D of the chunk
    template <int D>
    static constexpr uint32_t all_lo() { return (uint32_t)(kAll << D); }
    template <int D>
    static constexpr uint32_t all_hi() { return (uint32_t)((kAll << D) >> 32); }
};

// A chunk's frame: the Q planes and the "base exists" plane, W words each.
struct RwcF {
    uint32_t l0, l1, h0, h1, v0, v1;
};

// Column D of the chunk (before the row end); tl/th: the R bits of D's
// quad of columns, spread by spread4; two holds 2 (a run-time value, so
// that the move by one bit is a multiply on the FMA pipe).  The column's
// rows are S & ~(Q lo ^ R lo) & ~(Q hi ^ R hi): one three-input logic op
// per plane and word.  If none survives, the last surviving row met its
// obstacle here: counted, and every row is alive again at column D + 1,
// which is bit pattern all << D one move before.
template <int E, bool EDGE, int D>
SS_HD void rwc_column(uint32_t &s0, uint32_t &s1, int &count, const RwcF &f,
                      uint32_t tl, uint32_t th, uint32_t two)
{
    using Fr = RwcFrame<E>;
    if constexpr (D > 0) {  // one column right: every row one bit up
        if constexpr (Fr::W == 2)
            s1 = funnel_l(s0, s1, 1);
        s0 = s0 * two;
    }
    const uint32_t bl = byte_sign<D & 3>(tl);
    const uint32_t bh = byte_sign<D & 3>(th);
    uint32_t t0 = s0 & ~(f.l0 ^ bl);
    t0 &= ~(f.h0 ^ bh);
    if (EDGE)
        t0 &= f.v0;
    bool z;
    if constexpr (Fr::W == 2) {
        uint32_t t1 = s1 & ~(f.l1 ^ bl);
        t1 &= ~(f.h1 ^ bh);
        if (EDGE)
            t1 &= f.v1;
        z = (t0 | t1) == 0u;
        s1 = z ? Fr::template all_hi<D>() : t1;
    } else {
        z = t0 == 0u;
    }
    count += z;
    s0 = z ? Fr::template all_lo<D>() : t0;
}

// Columns I of the chunk for I in the sequence; with TAIL, only those
// with I < live (the row end's partial chunk: a uniform test per column).
template <int E, bool EDGE, bool TAIL, int... I>
SS_HD void rwc_columns(uint32_t &s0, uint32_t &s1, int &count,
                       const RwcF &f, uint32_t l0, uint32_t h0, uint32_t l1,
                       uint32_t h1, uint32_t two, int live,
                       std::integer_sequence<int, I...>)
{
    ((!TAIL || I < live
          ? rwc_column<E, EDGE, I>(s0, s1, count, f, I < 4 ? l0 : l1,
                                   I < 4 ? h0 : h1, two)
          : void()),
     ...);
}

// The chunk of columns D0 .. D0+KC-1 of the word (the first `live` of them
// with TAIL): its frame from the word's Q planes, the survivors moved into
// it (they sat at bits KC-1 .. KC-1+2E of the previous chunk's frame), and
// its columns.
template <int E, bool EDGE, int D0, bool TAIL = false>
SS_HD void rwc_chunk(uint32_t &s0, uint32_t &s1, int &count, const RwcQ &q,
                     uint32_t rlo, uint32_t rhi, uint32_t two, int live = 8)
{
    using Fr = RwcFrame<E>;
    constexpr int KC = Fr::KC;
    constexpr int O = D0 - E;  // frame bit 0 relative to the word
    RwcF f;
    f.l0 = rwc_window<O>(q.lo_p, q.lo_c, q.lo_n);
    f.h0 = rwc_window<O>(q.hi_p, q.hi_c, q.hi_n);
    f.v0 = EDGE ? rwc_window<O>(q.v_p, q.v_c, q.v_n) : 0u;
    if constexpr (Fr::W == 2) {
        f.l1 = rwc_window_up<O + 32>(q.lo_c, q.lo_n);
        f.h1 = rwc_window_up<O + 32>(q.hi_c, q.hi_n);
        f.v1 = EDGE ? rwc_window_up<O + 32>(q.v_c, q.v_n) : 0u;
        s0 = funnel_r(s0, s1, KC - 1);
        s1 >>= KC - 1;
    } else {
        f.l1 = f.h1 = f.v1 = 0u;
        s0 >>= KC - 1;
    }
    const uint32_t l0 = spread4(rlo >> D0), h0 = spread4(rhi >> D0);
    const uint32_t l1 = KC > 4 ? spread4(rlo >> (D0 + 4)) : 0u;
    const uint32_t h1 = KC > 4 ? spread4(rhi >> (D0 + 4)) : 0u;
    rwc_columns<E, EDGE, TAIL>(s0, s1, count, f, l0, h0, l1, h1, two, live,
                               std::make_integer_sequence<int, KC>{});
}

// Chunk D0 of the word at column base: the walk's result if it ends here
// (the row end, or the count past E), else -1.  A chunk is an edge chunk
// when one of its rows reads a query index below 0 or at/after m.
template <int E, int D0>
SS_HD int rwc_chunk_at(uint32_t &s0, uint32_t &s1, int &count,
                       const RwcQ &q, uint32_t rlo, uint32_t rhi, int base,
                       int m, uint32_t two)
{
    constexpr int KC = RwcFrame<E>::KC;
    const int c0 = base + D0;
    if (c0 + KC > m) {
        rwc_chunk<E, true, D0, true>(s0, s1, count, q, rlo, rhi, two,
                                     m - c0);
        return count <= E ? count : E + 1;
    }
    if (c0 < E || c0 + KC - 1 + E >= m)
        rwc_chunk<E, true, D0>(s0, s1, count, q, rlo, rhi, two);
    else
        rwc_chunk<E, false, D0>(s0, s1, count, q, rlo, rhi, two);
    return count > E ? E + 1 : -1;
}

// The word's chunks D0 = 0, KC, 2 KC, ... in order until one ends the walk.
template <int E, int... J>
SS_HD int rwc_word(uint32_t &s0, uint32_t &s1, int &count, const RwcQ &q,
                   uint32_t rlo, uint32_t rhi, int base, int m,
                   uint32_t two, std::integer_sequence<int, J...>)
{
    constexpr int KC = RwcFrame<E>::KC;
    int res = -1;
    ((res < 0 ? (res = rwc_chunk_at<E, J * KC>(s0, s1, count, q, rlo, rhi,
                                                base, m, two),
                 0)
              : 0),
     ...);
    return res;
}

// Route one pair of length m with threshold E (1 <= E <= 31) in the frame
// form; returns min(count, E+1), equal to rw_route's.  Reads the Q words up
// to the one after the word being walked (planes k+1), as rw_route does.
// neg1 holds 0xffffffff (the multiplier 2 is derived from it at run time).
template <int E, class Seq>
SS_HD int rw_route_frame(const Seq &Qs, const Seq &Rs, int m, uint32_t neg1)
{
    using Fr = RwcFrame<E>;
    constexpr int KC = Fr::KC;
    const uint32_t two = 4u + neg1 + neg1;
    const int W32 = (m + 31) >> 5;
    RwcQ q;
    q.lo_p = q.hi_p = q.v_p = 0u;  // before the query: case 4
    Qs.planes(0, q.lo_c, q.hi_c);
    Qs.planes(1, q.lo_n, q.hi_n);
    q.v_c = mask_below(m);
    q.v_n = mask_below(m - 32);
    // every row alive at the first column: all rows at bits KC-1.. of a
    // frame one chunk back
    uint32_t s0 = Fr::template all_lo<KC - 1>();
    uint32_t s1 = Fr::template all_hi<KC - 1>();
    int count = 0;
    for (int k = 0; k < W32; ++k) {
        const int base = k << 5;
        uint32_t rlo, rhi;
        Rs.planes(k, rlo, rhi);
        const int res =
            rwc_word<E>(s0, s1, count, q, rlo, rhi, base, m, two,
                        std::make_integer_sequence<int, 32 / KC>{});
        if (res >= 0)
            return res;
        // slide the Q windows by one word
        q.lo_p = q.lo_c;
        q.hi_p = q.hi_c;
        q.v_p = q.v_c;
        q.lo_c = q.lo_n;
        q.hi_c = q.hi_n;
        q.v_c = q.v_n;
        Qs.planes(k + 2, q.lo_n, q.hi_n);
        q.v_n = mask_below(m - 32 * (k + 2));
    }
    return count <= E ? count : E + 1;
}

// The column walk for threshold E (1 <= E <= 31): the frame form, except
// where its chunk would be two columns (E = 15 and 31), whose chunk set-up
// costs more than it saves (A/B on GB300 at 100 bp: E = 15 2.00 against
// 1.64 ms, E = 31 3.49 against 2.93 ms per 30M pairs).
template <int E, class Seq>
SS_HD int rw_route_cols(const Seq &Qs, const Seq &Rs, int m, uint32_t neg1)
{
    if constexpr (RwcFrame<E>::KC == 2)
        return rw_route_qshift<E>(Qs, Rs, m);
    else
        return rw_route_frame<E>(Qs, Rs, m, neg1);
}

}  // namespace ssk
