// ss_unequal.cuh -- pairs of different lengths (Section 2.4's correction).
//
// The maze has one column per reference base (Eq. 1 compares R[j]) and the
// 2E+1 rows of Eq. 1; a cell whose query index leaves 1..mQ is case 4.
// With equal lengths such cells are obstacles, as in rw_route.  When the
// lengths differ, the paper deducts the leading and trailing obstacles that
// case 4 causes: here those cells -- before the query's first base or after
// its last, on every diagonal -- are free, so the net passes the sequences'
// overhanging ends at no cost.
//
// rw_route2 is rw_route with separate query and reference lengths: the
// "query base exists" plane comes from mQ and is ANDed into the mismatch
// word (free) instead of ORed in inverted (obstacle).
#pragma once
#include <cstdint>
#include <type_traits>

#include "ss_device.cuh"
#include "ss_rwc.cuh"

namespace ssk {

// Rows needed by a pair, or -1 when the answer is 0 obstacles without
// routing (no reference column, or, with different lengths, a row of the
// 2E+1 that compares no base at all: every cell of it is free).
SS_HD int unequal_rows(int mQ, int mR, int E)
{
    if (mR == 0)
        return -1;
    if (mQ == mR)
        return E < mR - 1 ? E : mR - 1;
    const int mmin = mQ < mR ? mQ : mR;
    return E >= mmin ? -1 : E;
}

template <int EMAX, class Seq>
SS_HD int rw_route2(const Seq &Qs, int mQ, const Seq &Rs, int mR, int E,
                    uint32_t neg1)
{
    constexpr int NR = 2 * EMAX + 1;
    using RowBits = typename std::conditional<(NR <= 32), uint32_t,
                                              uint64_t>::type;
    const bool free_ends = mQ != mR;
    const int W32 = (mR + 31) >> 5;
    uint32_t Z[NR];
    RowBits deadbits = 0;
    uint32_t qlo_p = 0u, qhi_p = 0u, qlo_c, qhi_c, qlo_n, qhi_n;
    Qs.planes(0, qlo_c, qhi_c);
    Qs.planes(1, qlo_n, qhi_n);
    int count = 0;
    bool finished = false;
    for (int k = 0; k < W32 && !finished; ++k) {
        const int base = k << 5;
        uint32_t rlo, rhi;
        Rs.planes(k, rlo, rhi);
        const bool edge = (k == 0) || (base + 32 + EMAX > mQ);
        // query-base-exists plane around word k (bits of query indices
        // 0..mQ-1), shifted with each row like the query
        const uint32_t v_p = k == 0 ? 0u : mask_below(mQ - base + 32);
        const uint32_t v_c = mask_below(mQ - base);
        const uint32_t v_n = mask_below(mQ - base - 32);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int s = r - EMAX;
            uint32_t ql, qh;
            if (s >= 0) {
                ql = funnel_r(qlo_c, qlo_n, s);
                qh = funnel_r(qhi_c, qhi_n, s);
            } else {
                ql = funnel_l(qlo_p, qlo_c, -s);
                qh = funnel_l(qhi_p, qhi_c, -s);
            }
            uint32_t z = (ql ^ rlo) | (qh ^ rhi);
            if (edge) {
                const uint32_t qv = s >= 0 ? funnel_r(v_c, v_n, s)
                                           : funnel_l(v_p, v_c, -s);
                z = free_ends ? (z & qv) : (z | ~qv);
            }
            if (s > E || -s > E)
                z = 0xffffffffu;  // row outside this pair's 2E+1
            Z[r] = z;
        }
        uint32_t M = 0xffffffffu;
        for (;;) {
            uint32_t A = 0xffffffffu;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const uint32_t x =
                    (Z[r] & M) |
                    (0u - (uint32_t)((deadbits >> r) & (RowBits)1));
                A &= x | (x * neg1);
            }
            if (A == 0u) {
                RowBits d = deadbits;
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    d |= (RowBits)((Z[r] & M) != 0u) << r;
                deadbits = d;
                break;
            }
            deadbits = 0;
            const int e = base + ffs32(A) - 1;
            if (e >= mR) {
                finished = true;
                break;
            }
            if (++count > E) {
                finished = true;
                break;
            }
            const int c = e + 1;
            if (c >= base + 32)
                break;
            M = 0xffffffffu << (c - base);
        }
        qlo_p = qlo_c;
        qhi_p = qhi_c;
        qlo_c = qlo_n;
        qhi_c = qhi_n;
        Qs.planes(k + 2, qlo_n, qhi_n);
    }
    return count;
}

// rw_route2 walked one column at a time (EMAX <= 15), as rw_route_cols
// walks the equal-length greedy: the 2 EMAX + 1 rows in one word, the
// pair's own 2E + 1 of them set in kAll, one column per reference base.
// In a chunk where a row reads a query index outside 0..mQ-1, a cell is an
// obstacle iff (in range and mismatched) or (out of range and the lengths
// are equal): one three-input op with the per-pair mask fe (all ones when
// the ends are free), so the warp's threads need not agree on it.
template <int EMAX, bool EDGE, int D>
SS_HD void uqc_column(uint32_t &S, int &count, const RwcQ &q, uint32_t tl,
                      uint32_t th, uint32_t kAll, uint32_t fe)
{
    constexpr int O = D - EMAX;  // Q bit of row 0 relative to the word
    const uint32_t xl =
        rwc_window<O>(q.lo_p, q.lo_c, q.lo_n) ^ byte_sign<D & 3>(tl);
    const uint32_t xh =
        rwc_window<O>(q.hi_p, q.hi_c, q.hi_n) ^ byte_sign<D & 3>(th);
    if (EDGE) {
        const uint32_t qv = rwc_window<O>(q.v_p, q.v_c, q.v_n);
        const uint32_t mis = xl | xh;
        S &= ~((qv & mis) | (~qv & ~fe));
    } else {
        S &= ~xl;
        S &= ~xh;
    }
    const bool z = S == 0u;  // the last free row met its obstacle here
    count += z;
    S = z ? kAll : S;
}

template <int EMAX, bool EDGE, int D0, bool TAIL, int... I>
SS_HD void uqc_columns(uint32_t &S, int &count, const RwcQ &q, uint32_t l0,
                       uint32_t h0, uint32_t l1, uint32_t h1, uint32_t kAll,
                       uint32_t fe, int live, std::integer_sequence<int, I...>)
{
    ((!TAIL || I < live
          ? uqc_column<EMAX, EDGE, D0 + I>(S, count, q, I < 4 ? l0 : l1,
                                           I < 4 ? h0 : h1, kAll, fe)
          : void()),
     ...);
}

// Chunk D0 (8 columns) of the word at column base: the result if the walk
// ends here (the reference's end, or the count past E), else -1.
template <int EMAX, int D0>
SS_HD int uqc_chunk_at(uint32_t &S, int &count, const RwcQ &q, uint32_t rlo,
                       uint32_t rhi, uint32_t kAll, uint32_t fe, int base,
                       int mQ, int mR, int Er, int E)
{
    const int c0 = base + D0;
    const uint32_t l0 = spread4(rlo >> D0), h0 = spread4(rhi >> D0);
    const uint32_t l1 = spread4(rlo >> (D0 + 4));
    const uint32_t h1 = spread4(rhi >> (D0 + 4));
    const auto cols = std::make_integer_sequence<int, 8>{};
    if (c0 + 8 > mR) {  // the reference's end
        uqc_columns<EMAX, true, D0, true>(S, count, q, l0, h0, l1, h1, kAll,
                                          fe, mR - c0, cols);
        return count <= E ? count : E + 1;
    }
    if (c0 < Er || c0 + 7 + Er >= mQ)
        uqc_columns<EMAX, true, D0, false>(S, count, q, l0, h0, l1, h1, kAll,
                                           fe, 8, cols);
    else
        uqc_columns<EMAX, false, D0, false>(S, count, q, l0, h0, l1, h1,
                                            kAll, fe, 8, cols);
    return count > E ? E + 1 : -1;
}

// rw_route2's result, walked one column at a time (EMAX <= 15).
template <int EMAX, class Seq>
SS_HD int rw_route2_cols(const Seq &Qs, int mQ, const Seq &Rs, int mR,
                         int E)
{
    static_assert(EMAX >= 1 && EMAX <= 15, "2 EMAX + 1 rows in one word");
    const int Er = E < EMAX ? E : EMAX;  // rows past EMAX read no base
    const uint32_t kAll = ((2u << (2 * Er)) - 1u) << (EMAX - Er);
    const uint32_t fe = mQ != mR ? 0xffffffffu : 0u;
    const int W32 = (mR + 31) >> 5;
    RwcQ q;
    q.lo_p = q.hi_p = q.v_p = 0u;  // before the query
    Qs.planes(0, q.lo_c, q.hi_c);
    Qs.planes(1, q.lo_n, q.hi_n);
    q.v_c = mask_below(mQ);
    q.v_n = mask_below(mQ - 32);
    uint32_t S = kAll;
    int count = 0;
    for (int k = 0; k < W32; ++k) {
        const int base = k << 5;
        uint32_t rlo, rhi;
        Rs.planes(k, rlo, rhi);
        int res;
        if ((res = uqc_chunk_at<EMAX, 0>(S, count, q, rlo, rhi, kAll, fe,
                                         base, mQ, mR, Er, E)) >= 0 ||
            (res = uqc_chunk_at<EMAX, 8>(S, count, q, rlo, rhi, kAll, fe,
                                         base, mQ, mR, Er, E)) >= 0 ||
            (res = uqc_chunk_at<EMAX, 16>(S, count, q, rlo, rhi, kAll, fe,
                                          base, mQ, mR, Er, E)) >= 0 ||
            (res = uqc_chunk_at<EMAX, 24>(S, count, q, rlo, rhi, kAll, fe,
                                          base, mQ, mR, Er, E)) >= 0)
            return res;
        q.lo_p = q.lo_c;
        q.hi_p = q.hi_c;
        q.v_p = q.v_c;
        q.lo_c = q.lo_n;
        q.hi_c = q.hi_n;
        q.v_c = q.v_n;
        Qs.planes(k + 2, q.lo_n, q.hi_n);
        q.v_n = mask_below(mQ - 32 * (k + 2));
    }
    return count <= E ? count : E + 1;
}

// The routine of the row class EMAX (rows 2 EMAX + 1): row-wise for 7 and
// 63 rows, the column walk for 15 and 31.
template <int EMAX, class Seq>
SS_HD int unequal_route(const Seq &q, int mQ, const Seq &r, int mR, int E,
                        uint32_t neg1)
{
    if constexpr (EMAX >= 7 && EMAX <= 15)
        return rw_route2_cols<EMAX>(q, mQ, r, mR, E);
    else
        return rw_route2<EMAX>(q, mQ, r, mR, E, neg1);
}

// Predicted routing cost of a staged pair of different lengths: the fewest
// mismatches over reference columns 16..31 on any diagonal of the pair's
// band, |s| <= min(E, 16).  A read inside a reference window with a
// random flank of o bases matches on diagonal -o, away from the centre;
// columns 16..31 read query bases (not the flank) on every such diagonal,
// so each diagonal counts 16 comparisons.  Words 0..3 of the query and
// 0..1 of the reference are read (whatever follows a short pair's words in
// its slot only blurs the estimate).
SS_HD int uq_cost_key(const uint32_t *sq, const uint32_t *sr, int E)
{
    uint32_t qlo, qhi, qlo_n, qhi_n, rlo, rhi;
    planes_of(sq[0], sq[1], qlo, qhi);
    planes_of(sq[2], sq[3], qlo_n, qhi_n);
    planes_of(sr[0], sr[1], rlo, rhi);
    const int band = E < 16 ? E : 16;
    int k = 16;
    for (int s = -band; s <= band; ++s) {
        uint32_t ql, qh;
        if (s >= 0) {
            ql = funnel_r(qlo, qlo_n, (uint32_t)s);
            qh = funnel_r(qhi, qhi_n, (uint32_t)s);
        } else {
            ql = qlo << -s;
            qh = qhi << -s;
        }
        const uint32_t mis = ((ql ^ rlo) | (qh ^ rhi)) & 0xffff0000u;
#ifdef __CUDA_ARCH__
        k = imin(k, __popc(mis));
#else
        k = imin(k, __builtin_popcount(mis));
#endif
    }
    return k;
}

// ---- exact-E routines (one threshold for every pair of the launch) ------

// Column D of a chunk in the frame form (ss_rwc.cuh) for a pair of
// different lengths: where a row can leave the query (EDGE) a cell is an
// obstacle iff it is in range and mismatched, or out of range with equal
// lengths (nfe: all ones when the lengths are equal, else 0).
template <int E, bool EDGE, int D>
SS_HD void uqf_column(uint32_t &s0, int &count, const RwcF &f, uint32_t tl,
                      uint32_t th, uint32_t two, uint32_t nfe)
{
    using Fr = RwcFrame<E>;
    if constexpr (D > 0)
        s0 = s0 * two;  // one column right: every row one bit up
    const uint32_t bl = byte_sign<D & 3>(tl);
    const uint32_t bh = byte_sign<D & 3>(th);
    uint32_t t0;
    if (EDGE) {
        const uint32_t mis = (f.l0 ^ bl) | (f.h0 ^ bh);
        t0 = s0 & ~((f.v0 & mis) | (~f.v0 & nfe));
    } else {
        t0 = s0 & ~(f.l0 ^ bl);
        t0 &= ~(f.h0 ^ bh);
    }
    const bool z = t0 == 0u;  // the last free row met its obstacle here
    count += z;
    s0 = z ? Fr::template all_lo<D>() : t0;
}

template <int E, bool EDGE, bool TAIL, int... I>
SS_HD void uqf_columns(uint32_t &s0, int &count, const RwcF &f, uint32_t l0,
                       uint32_t h0, uint32_t l1, uint32_t h1, uint32_t two,
                       uint32_t nfe, int live, std::integer_sequence<int, I...>)
{
    ((!TAIL || I < live
          ? uqf_column<E, EDGE, I>(s0, count, f, I < 4 ? l0 : l1,
                                   I < 4 ? h0 : h1, two, nfe)
          : void()),
     ...);
}

// The chunk of columns D0 .. D0+KC-1 of the reference word (the first
// `live` of them with TAIL), as rwc_chunk with one survivor word.
template <int E, bool EDGE, int D0, bool TAIL = false>
SS_HD void uqf_chunk(uint32_t &s0, int &count, const RwcQ &q, uint32_t rlo,
                     uint32_t rhi, uint32_t two, uint32_t nfe, int live = 8)
{
    using Fr = RwcFrame<E>;
    static_assert(Fr::W == 1 && Fr::KC >= 4, "one survivor word");
    constexpr int KC = Fr::KC;
    constexpr int O = D0 - E;
    RwcF f;
    f.l0 = rwc_window<O>(q.lo_p, q.lo_c, q.lo_n);
    f.h0 = rwc_window<O>(q.hi_p, q.hi_c, q.hi_n);
    f.v0 = EDGE ? rwc_window<O>(q.v_p, q.v_c, q.v_n) : 0u;
    f.l1 = f.h1 = f.v1 = 0u;
    s0 >>= KC - 1;
    const uint32_t l0 = spread4(rlo >> D0), h0 = spread4(rhi >> D0);
    const uint32_t l1 = KC > 4 ? spread4(rlo >> (D0 + 4)) : 0u;
    const uint32_t h1 = KC > 4 ? spread4(rhi >> (D0 + 4)) : 0u;
    uqf_columns<E, EDGE, TAIL>(s0, count, f, l0, h0, l1, h1, two, nfe, live,
                               std::make_integer_sequence<int, KC>{});
}

// Chunk D0 of the reference word at column base: the result if the walk
// ends here (the reference's end, or the count past E), else -1.
template <int E, int D0>
SS_HD int uqf_chunk_at(uint32_t &s0, int &count, const RwcQ &q, uint32_t rlo,
                       uint32_t rhi, int base, int mQ, int mR, uint32_t two,
                       uint32_t nfe)
{
    constexpr int KC = RwcFrame<E>::KC;
    const int c0 = base + D0;
    if (c0 + KC > mR) {
        uqf_chunk<E, true, D0, true>(s0, count, q, rlo, rhi, two, nfe,
                                     mR - c0);
        return count <= E ? count : E + 1;
    }
    if (c0 < E || c0 + KC - 1 + E >= mQ)
        uqf_chunk<E, true, D0>(s0, count, q, rlo, rhi, two, nfe);
    else
        uqf_chunk<E, false, D0>(s0, count, q, rlo, rhi, two, nfe);
    return count > E ? E + 1 : -1;
}

template <int E, int... J>
SS_HD int uqf_word(uint32_t &s0, int &count, const RwcQ &q, uint32_t rlo,
                   uint32_t rhi, int base, int mQ, int mR, uint32_t two,
                   uint32_t nfe, std::integer_sequence<int, J...>)
{
    constexpr int KC = RwcFrame<E>::KC;
    int res = -1;
    ((res < 0 ? (res = uqf_chunk_at<E, J * KC>(s0, count, q, rlo, rhi, base,
                                                mQ, mR, two, nfe),
                 0)
              : 0),
     ...);
    return res;
}

// rw_route2's result for threshold E (5 <= E <= 14), walked in the frame
// form: one column per reference base, the 2E+1 rows in one word.
template <int E, class Seq>
SS_HD int rw_route2_frame(const Seq &Qs, int mQ, const Seq &Rs, int mR,
                          uint32_t neg1)
{
    using Fr = RwcFrame<E>;
    constexpr int KC = Fr::KC;
    const uint32_t two = 4u + neg1 + neg1;
    const uint32_t nfe = mQ == mR ? 0xffffffffu : 0u;
    const int W32 = (mR + 31) >> 5;
    RwcQ q;
    q.lo_p = q.hi_p = q.v_p = 0u;  // before the query
    Qs.planes(0, q.lo_c, q.hi_c);
    Qs.planes(1, q.lo_n, q.hi_n);
    q.v_c = mask_below(mQ);
    q.v_n = mask_below(mQ - 32);
    uint32_t s0 = Fr::template all_lo<KC - 1>();
    int count = 0;
    for (int k = 0; k < W32; ++k) {
        const int base = k << 5;
        uint32_t rlo, rhi;
        Rs.planes(k, rlo, rhi);
        const int res =
            uqf_word<E>(s0, count, q, rlo, rhi, base, mQ, mR, two, nfe,
                        std::make_integer_sequence<int, 32 / KC>{});
        if (res >= 0)
            return res;
        q.lo_p = q.lo_c;
        q.hi_p = q.hi_c;
        q.v_p = q.v_c;
        q.lo_c = q.lo_n;
        q.hi_c = q.hi_n;
        q.v_c = q.v_n;
        Qs.planes(k + 2, q.lo_n, q.hi_n);
        q.v_n = mask_below(mQ - 32 * (k + 2));
    }
    return count <= E ? count : E + 1;
}

// The routine for one threshold E shared by every pair of a launch:
// row-wise with exactly 2E+1 rows up to E = 4 and above 15, the frame-form
// column walk for 5..14, the column walk with shifted query windows at 15.
template <int E, class Seq>
SS_HD int unequal_route_exact(const Seq &q, int mQ, const Seq &r, int mR,
                              uint32_t neg1)
{
    if constexpr (E >= 5 && E <= 14)
        return rw_route2_frame<E>(q, mQ, r, mR, neg1);
    else if constexpr (E == 15)
        return rw_route2_cols<15>(q, mQ, r, mR, E);
    else
        return rw_route2<E>(q, mQ, r, mR, E, neg1);
}

}  // namespace ssk
