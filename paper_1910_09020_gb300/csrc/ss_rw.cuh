// ss_rw.cuh -- K3a: SneakySnake, one thread per pair, maze rows bit-parallel
// along the columns ("row-wise").
//
// Method (Section 2.3-2.4): row i of the chip maze Z compares R[j] with the
// Q base on diagonal s = i - (E+1) (Eq. 1: rows 1..E are s = -1..-E, row E+1
// is s = 0, rows E+2..2E+1 are s = 1..E); entries whose Q index leaves 1..m
// are obstacles.  From a checkpoint, the longest run of zeros over the 2E+1
// rows is taken, the obstacle ending it is counted and the checkpoint moves
// past it, until the row end is reached or the count exceeds E.
//
// GB300 mapping: each thread holds, for the 32-column word k it is routing
// through, the maze row words Z_s (one register each, built with one funnel
// shift per bit plane and two logic ops: the maze is built lazily word by
// word, as in the implicit maze of Section 2.4).  The longest run from
// checkpoint c needs no per-row bit scan: with x_s = Z_s masked to columns
// >= c, x_s | -x_s sets every bit at or above row s's first obstacle, so the
// AND over rows has its lowest set bit at max_s(first obstacle) -- the end of
// the longest escape segment -- found with one find-first per iteration.
// When a run crosses into the next word, the rows that already met an
// obstacle since c are kept in a bitmask and count as all-obstacle rows
// until the next obstacle is found, so runs spanning words are exact.
//
// Two launch forms share rw_route():
//  * k_rw_uniform<E>: the plain launch (uniform m and E).  A CTA stages its
//    pairs' packed words in shared memory, transposed (word i of the CTA's
//    pair t at [i * ld + t], ld = T + 1) so per-thread reads are
//    conflict-free; results are written coalesced.
//  * k_rw_bucket<EMAX>: persistent launch over one bucket of a mixed batch
//    (runtime E <= EMAX, any m); each thread reads its pair straight from
//    global memory (contiguous words, L1-cached).  Rows with |s| > E are
//    all-obstacle rows, which never bound the longest run.
#pragma once
#include <cstdint>

#include "ss_device.cuh"

namespace ssk {

// Packed words of one sequence, transposed in shared memory (word i at
// s[i * ld]).
struct SmemSeq {
    const uint32_t *s;
    int ld;
    int w16;
    SS_HD void planes(int k, uint32_t &lo, uint32_t &hi) const
    {
        const int i = 2 * k;
        const uint32_t p0 = i < w16 ? s[i * ld] : 0u;
        const uint32_t p1 = i + 1 < w16 ? s[(i + 1) * ld] : 0u;
        planes_of(p0, p1, lo, hi);
    }
};

// Packed words of one sequence in global memory.
struct GlobalSeq {
    const uint32_t *g;
    int w16;
    SS_HD void planes(int k, uint32_t &lo, uint32_t &hi) const
    {
        const int i = 2 * k;
        const uint32_t p0 = i < w16 ? ldg(g + i) : 0u;
        const uint32_t p1 = i + 1 < w16 ? ldg(g + i + 1) : 0u;
        planes_of(p0, p1, lo, hi);
    }
};

// Route one pair of length m with threshold E (E == EMAX when EXACT);
// returns min(count, E+1).  Rows |s| > min(E, EMAX) are never built.
template <int EMAX, bool EXACT, class Seq>
SS_HD int rw_route(const Seq &Qs, const Seq &Rs, int m, int E)
{
    constexpr int NR = 2 * EMAX + 1;
    const int W32 = (m + 31) >> 5;
    uint32_t Z[NR];
    uint64_t deadbits = 0;  // rows that met an obstacle since c (crossing)

    uint32_t qlo_p = 0u, qhi_p = 0u, qlo_c, qhi_c, qlo_n, qhi_n;
    Qs.planes(0, qlo_c, qhi_c);
    Qs.planes(1, qlo_n, qhi_n);

    int count = 0;
    bool finished = false;
    for (int k = 0; k < W32 && !finished; ++k) {
        const int base = k << 5;
        uint32_t rlo, rhi;
        Rs.planes(k, rlo, rhi);
        const bool edge = (k == 0) || (base + 32 + EMAX > m);
        // Eq. 1 for the 32 columns of word k, every row.
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
                // case 4: Q index below 1 (word 0 only) or above m; columns
                // past m act as a sentinel (tested as "reached the end").
                if (s < 0)
                    z |= mask_below(-s - base);
                z |= mask_from((s > 0 ? m - s : m) - base);
            }
            if (!EXACT && (s > E || -s > E))
                z = 0xffffffffu;  // row outside this pair's 2E+1
            Z[r] = z;
        }
        // Greedy routing inside word k (checkpoint c <= base on entry).
        uint32_t M = 0xffffffffu;  // columns >= checkpoint
        for (;;) {
            uint32_t A = 0xffffffffu;
            if (deadbits) {
                // runs continued from the previous word: rows that already
                // met an obstacle since the checkpoint do not count
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const uint32_t x = (Z[r] & M) |
                                       (0u - (uint32_t)((deadbits >> r) & 1u));
                    A &= x | (0u - x);
                }
            } else {
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const uint32_t x = Z[r] & M;
                    A &= x | (0u - x);
                }
            }
            if (A == 0u) {
                // a live row runs past the word end: remember the others
                uint64_t d = deadbits;
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    d |= (uint64_t)((Z[r] & M) != 0u) << r;
                deadbits = d;
                break;
            }
            deadbits = 0;  // an obstacle ends every run: fresh checkpoint
            const int e = base + ffs32(A) - 1;  // end of the escape segment
            if (e >= m) {                       // reached the destination
                finished = true;
                break;
            }
            ++count;                            // its obstacle
            if (count > E) {                    // delay exceeds E: reject
                finished = true;
                break;
            }
            const int c = e + 1;                // new checkpoint
            if (c >= base + 32)
                break;
            M = 0xffffffffu << (c - base);
        }
        // slide the Q window by one word
        qlo_p = qlo_c;
        qhi_p = qhi_c;
        qlo_c = qlo_n;
        qhi_c = qhi_n;
        Qs.planes(k + 2, qlo_n, qhi_n);
    }
    return count;
}

struct RwUniformArgs {
    const uint32_t *reads;  // packed, pair p at word p * w16
    const uint32_t *refs;
    int64_t n;
    int32_t m;
    int32_t w16;
    uint32_t w16_magic;
    uint8_t *acc;
    int32_t *obs;
};

// Plain launch: uniform m and E, one thread per pair, one CTA per T pairs.
template <int E>
__global__ void __launch_bounds__(128)
    k_rw_uniform(const RwUniformArgs a)
{
    extern __shared__ uint32_t smem[];
    const int T = blockDim.x;
    const int ld = T + 1;
    const int64_t p0 = (int64_t)blockIdx.x * T;
    const int64_t left = a.n - p0;
    const int np = left < T ? (int)left : T;
    uint32_t *sQ = smem;
    uint32_t *sR = smem + (size_t)a.w16 * ld;
    const int total = np * a.w16;
    const uint32_t *gq = a.reads + p0 * a.w16;
    const uint32_t *gr = a.refs + p0 * a.w16;
    for (int idx = threadIdx.x; idx < total; idx += T) {
        const uint32_t t = fast_div((uint32_t)idx, (uint32_t)a.w16,
                                    a.w16_magic);
        const uint32_t i = (uint32_t)idx - t * (uint32_t)a.w16;
        sQ[i * ld + t] = __ldg(gq + idx);
        sR[i * ld + t] = __ldg(gr + idx);
    }
    __syncthreads();
    if (threadIdx.x < np) {
        const SmemSeq q{sQ + threadIdx.x, ld, a.w16};
        const SmemSeq r{sR + threadIdx.x, ld, a.w16};
        const int cnt = rw_route<E, true>(q, r, a.m, E);
        a.acc[p0 + threadIdx.x] = (uint8_t)(cnt <= E);
        a.obs[p0 + threadIdx.x] = cnt;
    }
}

}  // namespace ssk
