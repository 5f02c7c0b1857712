// ss_submaze.cuh -- Snake-on-Chip's decomposition (Section 2.5) on the GPU:
// the maze is cut into sub-mazes of t consecutive columns, each routed
// independently by the greedy of Section 2.4 (at most y escape segments per
// sub-maze), and their obstacle counts are summed.  The paper notes this can
// only underestimate the full count; it is an opt-in approximate mode, not
// the exact filter.
#pragma once
#include <cstdint>
#include <type_traits>

#include "ss_device.cuh"
#include "ss_rw.cuh"
#include "ss_rwc.cuh"

namespace ssk {

// Sum of the t-column sub-mazes' counts (each at most y), stopped once it
// exceeds E; returns min(total, E+1).  Sub-mazes are routed in order -- the
// same loop for every thread of a warp, as t is uniform -- and each keeps
// its own checkpoint: sub-maze [a, b) starts fresh at a; a run whose first
// obstacle lies at or past b reaches the sub-maze's last column and ends it
// without an obstacle; it holds at most min(y, E + 1 - total) obstacles.
// The maze rows of a 32-column word are built once and kept while the
// following sub-mazes stay in that word.
template <int EMAX, class Seq>
SS_HD int submaze_route(const Seq &Qs, const Seq &Rs, int m, int E, int t,
                        int y, uint32_t neg1)
{
    constexpr int NR = 2 * EMAX + 1;
    using RowBits = typename std::conditional<(NR <= 32), uint32_t,
                                              uint64_t>::type;
    uint32_t Z[NR];
    int kz = -1;  // word whose rows Z holds
    int total = 0;
    for (int a = 0; a < m && total <= E; a = t < m - a ? a + t : m) {
        const int b = t < m - a ? a + t : m;
        const int cap = y < E + 1 - total ? y : E + 1 - total;
        int c = a, seg = 0;
        RowBits deadbits = 0;
        for (;;) {
            const int k = c >> 5;
            const int base = k << 5;
            if (k != kz) {  // Eq. 1 for the 32 columns of word k
                uint32_t qlo_p = 0u, qhi_p = 0u, qlo_c, qhi_c, qlo_n, qhi_n;
                if (k > 0)
                    Qs.planes(k - 1, qlo_p, qhi_p);
                Qs.planes(k, qlo_c, qhi_c);
                Qs.planes(k + 1, qlo_n, qhi_n);
                uint32_t rlo, rhi;
                Rs.planes(k, rlo, rhi);
                const bool lo_edge = k == 0;
                const bool hi_edge = base + 32 + EMAX > m;
                const uint32_t v_c = mask_below(m - base);
                const uint32_t v_n = mask_below(m - base - 32);
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
                    if (s < 0 && lo_edge)
                        z |= ~funnel_l(0u, v_c, -s);
                    else if (s > 0 && hi_edge)
                        z |= ~funnel_r(v_c, v_n, s);
                    if (s > E || -s > E)
                        z = 0xffffffffu;  // row outside this pair's 2E+1
                    Z[r] = z;
                }
                kz = k;
            }
            const uint32_t M = 0xffffffffu << (c - base);
            uint32_t A = 0xffffffffu;
            if (deadbits) {
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const uint32_t x =
                        (Z[r] & M) |
                        (0u - (uint32_t)((deadbits >> r) & (RowBits)1));
                    A &= x | (x * neg1);
                }
            } else {
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const uint32_t x = Z[r] & M;
                    A &= x | (x * neg1);
                }
            }
            if (A == 0u) {
                if (b <= base + 32)
                    break;  // a run reaches the sub-maze's last column
                // a live run leaves the word inside the sub-maze
                RowBits d = deadbits;
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    d |= (RowBits)((Z[r] & M) != 0u) << r;
                deadbits = d;
                c = base + 32;
                continue;
            }
            deadbits = 0;
            const int e = base + ffs32(A) - 1;
            if (e >= b)
                break;  // reached the sub-maze's destination
            ++total;
            if (++seg >= cap)
                break;
            c = e + 1;
            if (c >= b)
                break;
        }
    }
    return total < E + 1 ? total : E + 1;
}

// The same decomposition walked one column at a time (EMAX <= 15: the
// 2 EMAX + 1 rows in one word, the pair's own 2E + 1 of them set in
// kAll), as rw_route_cols walks the exact greedy.  S = the rows free of
// obstacles since the checkpoint; the column where S empties is the
// farthest first obstacle -- counted, at most y per sub-maze -- and S
// restarts; at a sub-maze's end (every t columns, the same column for all
// threads of a warp) its count is added to the total and S restarts.
template <int EMAX, bool EDGE, int D>
SS_HD void smc_column(uint32_t &S, int &seg, int &total, int &rem,
                      const RwcQ &q, uint32_t tl, uint32_t th, uint32_t kAll,
                      int t, int y)
{
    constexpr int O = D - EMAX;  // Q bit of row 0 relative to the word
    S &= ~(rwc_window<O>(q.lo_p, q.lo_c, q.lo_n) ^ byte_sign<D & 3>(tl));
    S &= ~(rwc_window<O>(q.hi_p, q.hi_c, q.hi_n) ^ byte_sign<D & 3>(th));
    if (EDGE)
        S &= rwc_window<O>(q.v_p, q.v_c, q.v_n);
    const bool z = S == 0u;  // the last free row met its obstacle here
    seg = imin(seg + (int)z, y);
    S = z ? kAll : S;
    if (--rem == 0) {  // the sub-maze's last column
        total += seg;
        seg = 0;
        S = kAll;
        rem = t;
    }
}

template <int EMAX, bool EDGE, int D0, bool TAIL, int... I>
SS_HD void smc_columns(uint32_t &S, int &seg, int &total, int &rem,
                       const RwcQ &q, uint32_t l0, uint32_t h0, uint32_t l1,
                       uint32_t h1, uint32_t kAll, int t, int y, int live,
                       std::integer_sequence<int, I...>)
{
    ((!TAIL || I < live
          ? smc_column<EMAX, EDGE, D0 + I>(S, seg, total, rem, q,
                                           I < 4 ? l0 : l1, I < 4 ? h0 : h1,
                                           kAll, t, y)
          : void()),
     ...);
}

// Chunk D0 (8 columns) of the word at column base: the result if the walk
// ends here (the row end, or the total past E), else -1.
template <int EMAX, int D0>
SS_HD int smc_chunk_at(uint32_t &S, int &seg, int &total, int &rem,
                       const RwcQ &q, uint32_t rlo, uint32_t rhi,
                       uint32_t kAll, int base, int m, int E, int t, int y)
{
    const int c0 = base + D0;
    const uint32_t l0 = spread4(rlo >> D0), h0 = spread4(rhi >> D0);
    const uint32_t l1 = spread4(rlo >> (D0 + 4));
    const uint32_t h1 = spread4(rhi >> (D0 + 4));
    const auto cols = std::make_integer_sequence<int, 8>{};
    if (c0 + 8 > m) {  // the row end
        smc_columns<EMAX, true, D0, true>(S, seg, total, rem, q, l0, h0, l1,
                                          h1, kAll, t, y, m - c0, cols);
        total += seg;
        return total <= E ? total : E + 1;
    }
    if (c0 < E || c0 + 7 + E >= m)
        smc_columns<EMAX, true, D0, false>(S, seg, total, rem, q, l0, h0,
                                           l1, h1, kAll, t, y, 8, cols);
    else
        smc_columns<EMAX, false, D0, false>(S, seg, total, rem, q, l0, h0,
                                            l1, h1, kAll, t, y, 8, cols);
    return total + seg > E ? E + 1 : -1;
}

// submaze_route's result, walked one column at a time (E <= EMAX <= 15).
template <int EMAX, class Seq>
SS_HD int submaze_route_cols(const Seq &Qs, const Seq &Rs, int m, int E,
                             int t, int y)
{
    static_assert(EMAX >= 1 && EMAX <= 15, "2 EMAX + 1 rows in one word");
    // the pair's rows; rows past m - 1 (E clamped to EMAX) are all case 4
    const int Er = E < EMAX ? E : EMAX;
    const uint32_t kAll = ((2u << (2 * Er)) - 1u) << (EMAX - Er);
    const int W32 = (m + 31) >> 5;
    RwcQ q;
    q.lo_p = q.hi_p = q.v_p = 0u;  // before the query: case 4
    Qs.planes(0, q.lo_c, q.hi_c);
    Qs.planes(1, q.lo_n, q.hi_n);
    q.v_c = mask_below(m);
    q.v_n = mask_below(m - 32);
    uint32_t S = kAll;
    int seg = 0, total = 0, rem = t;
    for (int k = 0; k < W32; ++k) {
        const int base = k << 5;
        uint32_t rlo, rhi;
        Rs.planes(k, rlo, rhi);
        int res;
        if ((res = smc_chunk_at<EMAX, 0>(S, seg, total, rem, q, rlo, rhi,
                                         kAll, base, m, E, t, y)) >= 0 ||
            (res = smc_chunk_at<EMAX, 8>(S, seg, total, rem, q, rlo, rhi,
                                         kAll, base, m, E, t, y)) >= 0 ||
            (res = smc_chunk_at<EMAX, 16>(S, seg, total, rem, q, rlo, rhi,
                                          kAll, base, m, E, t, y)) >= 0 ||
            (res = smc_chunk_at<EMAX, 24>(S, seg, total, rem, q, rlo, rhi,
                                          kAll, base, m, E, t, y)) >= 0)
            return res;
        q.lo_p = q.lo_c;
        q.hi_p = q.hi_c;
        q.v_p = q.v_c;
        q.lo_c = q.lo_n;
        q.hi_c = q.hi_n;
        q.v_c = q.v_n;
        Qs.planes(k + 2, q.lo_n, q.hi_n);
        q.v_n = mask_below(m - 32 * (k + 2));
    }
    total += seg;
    return total <= E ? total : E + 1;
}

}  // namespace ssk
