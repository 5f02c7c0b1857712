// ss_submaze.cuh -- Snake-on-Chip's decomposition (Section 2.5) on the GPU:
// the maze is cut into sub-mazes of t consecutive columns, each routed
// independently by the greedy of Section 2.4 (at most y escape segments per
// sub-maze), and their obstacle counts are summed.  The paper notes this can
// only underestimate the full count; it is an opt-in approximate mode, not
// the exact filter.
//
// rw_route_span is the row-wise routine of ss_rw.cuh restricted to columns
// [c0, c1): the checkpoint starts at c0, a run that reaches c1 ends the
// routing without an obstacle, and routing stops after ymax obstacles.
#pragma once
#include <cstdint>
#include <type_traits>

#include "ss_device.cuh"
#include "ss_rw.cuh"

namespace ssk {

template <int EMAX, class Seq>
SS_HD int rw_route_span(const Seq &Qs, const Seq &Rs, int m, int E, int c0,
                        int c1, int ymax, uint32_t neg1)
{
    constexpr int NR = 2 * EMAX + 1;
    using RowBits = typename std::conditional<(NR <= 32), uint32_t,
                                              uint64_t>::type;
    if (c0 >= c1 || ymax <= 0)
        return 0;
    uint32_t Z[NR];
    RowBits deadbits = 0;
    int k = c0 >> 5;
    uint32_t qlo_p = 0u, qhi_p = 0u, qlo_c, qhi_c, qlo_n, qhi_n;
    if (k > 0)
        Qs.planes(k - 1, qlo_p, qhi_p);
    Qs.planes(k, qlo_c, qhi_c);
    Qs.planes(k + 1, qlo_n, qhi_n);
    uint32_t M = 0xffffffffu << (c0 & 31);
    int count = 0;
    for (;; ++k) {
        const int base = k << 5;
        uint32_t rlo, rhi;
        Rs.planes(k, rlo, rhi);
        const bool edge = (k == 0) || (base + 32 + EMAX > m);
        const uint32_t v_p = k == 0 ? 0u : 0xffffffffu;
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
            uint32_t z;
            if (edge) {
                const uint32_t qv = s >= 0 ? funnel_r(v_c, v_n, s)
                                           : funnel_l(v_p, v_c, -s);
                z = (ql ^ rlo) | (qh ^ rhi) | ~qv;
            } else {
                z = (ql ^ rlo) | (qh ^ rhi);
            }
            if (s > E || -s > E)
                z = 0xffffffffu;  // row outside this pair's 2E+1
            Z[r] = z;
        }
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
                if (c1 <= base + 32)
                    return count;  // a run reaches the span's last column
                RowBits d = deadbits;
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    d |= (RowBits)((Z[r] & M) != 0u) << r;
                deadbits = d;
                M = 0xffffffffu;
                break;
            }
            deadbits = 0;
            const int e = base + ffs32(A) - 1;
            if (e >= c1)
                return count;  // reached the span's destination
            if (++count >= ymax)
                return count;
            const int c = e + 1;
            if (c >= c1)
                return count;
            if (c >= base + 32) {
                M = 0xffffffffu;
                break;
            }
            M = 0xffffffffu << (c - base);
        }
        qlo_p = qlo_c;
        qhi_p = qhi_c;
        qlo_c = qlo_n;
        qhi_c = qhi_n;
        Qs.planes(k + 2, qlo_n, qhi_n);
    }
}

// Sum of the t-column sub-mazes' counts (each at most y), stopped once it
// exceeds E; returns min(total, E+1).
template <int EMAX, class Seq>
SS_HD int submaze_route(const Seq &Qs, const Seq &Rs, int m, int E, int t,
                        int y, uint32_t neg1)
{
    int total = 0;
    for (int a = 0; a < m && total <= E; a += t) {
        const int b = a + t < m ? a + t : m;
        const int cap = y < E + 1 - total ? y : E + 1 - total;
        total += rw_route_span<EMAX>(Qs, Rs, m, E, a, b, cap, neg1);
    }
    return total < E + 1 ? total : E + 1;
}

}  // namespace ssk
