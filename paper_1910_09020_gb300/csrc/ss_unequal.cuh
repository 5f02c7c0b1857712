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

}  // namespace ssk
