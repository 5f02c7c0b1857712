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

}  // namespace ssk
