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
// word, as in the implicit maze of Section 2.4).  The longest run from the
// checkpoint needs no per-row bit scan: per row, one or two integer ops
// turn the row word into a mask whose AND (or OR) over rows has its lowest
// (highest) set bit at the farthest first obstacle -- the end of the
// longest escape segment -- found with one find-first per iteration
// (rw_word_smear below).  When a run crosses into the
// next word, the rows that already met an obstacle since the checkpoint
// are kept in a bitmask and count as blocked until the next obstacle is
// found, so runs spanning words are exact.
//
// Three launch forms share rw_route():
//  * k_rw_uniform<E>: the plain launch (uniform m and E, m <= 256).  Each
//    CTA routes a group of kRwGroup consecutive tiles of 128 pairs; a ring
//    of two shared-memory stages is filled by bulk asynchronous copies (one
//    per sequence per tile, completing on an mbarrier), so the next tiles'
//    HBM reads are in flight while the current tile is routed.  Groups, not
//    a persistent grid: the block scheduler hands out groups as SMs free
//    up, which balances the uneven routing cost of the groups.  Waits are
//    bounded: on timeout the CTA latches kStatusTimeout, drains its copies
//    in flight and returns.
//  * k_rw_staged<E>: the plain launch for longer reads; a CTA stages its
//    pairs' packed words in shared memory, transposed (word i of the CTA's
//    pair t at [i * ld + t], ld = T + 1), with no pipelining.
//  * k_rw_bucket<EMAX>: persistent launch over one bucket of a mixed batch
//    (runtime E <= EMAX, any m); each thread reads its pair straight from
//    global memory (contiguous words, L1-cached).  Rows with |s| > E are
//    all-obstacle rows, which never bound the longest run.
#pragma once
#include <cstdint>
#include <type_traits>

#include "ss_device.cuh"
#include "ss_rw_config.h"
#include "ss_rwc.cuh"

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

// Packed words of one sequence, contiguous in shared memory that extends at
// least 4 words past the sequence (the next pair's words or padding): no
// bounds check.  rw_route reads at most 4 words past ceil(m/16), and what it
// finds there only touches columns >= m (reference) or bits that the
// query-base-exists plane marks as case 4 (query).
struct SmemSeqPad {
    const uint32_t *s;
    SS_HD void planes(int k, uint32_t &lo, uint32_t &hi) const
    {
        planes_of(s[2 * k], s[2 * k + 1], lo, hi);
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

// Greedy routing inside one 32-column word (Section 2.4 steps 2-4) on its
// maze row words Z (row r = diagonal r - EMAX), entered with the
// checkpoint at or before the word start.  deadbits: rows that met an
// obstacle since that checkpoint (runs continued from the previous word);
// on return it holds them for the next word, or 0.  count and finished
// advance as the greedy does.
//
// Smear-AND (plain kernel E <= 4, bucketed kernel): with x_s = Z_s masked to
// columns >= c, x_s | -x_s sets every bit at or above row s's first
// obstacle, so the AND over rows has its lowest set bit at max_s(first
// obstacle): three operations per row and iteration, a find-first per
// iteration.  The word is entered at its first column (a checkpoint of the
// previous word is at most its end), so the first search needs no column
// mask, two operations per row; only it can carry blocked rows (a found
// obstacle clears them), so the later ones need no check for them.
template <int NR, class RowBits>
SS_HD void rw_word_smear(const uint32_t (&Z)[NR], RowBits &deadbits,
                         int base, int m, int E, int &count, bool &finished,
                         uint32_t neg1)
{
    uint32_t A = 0xffffffffu;
    if (deadbits) {
        // runs continued from the previous word: rows that already met an
        // obstacle since the checkpoint do not count
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const uint32_t x =
                Z[r] | (0u - (uint32_t)((deadbits >> r) & (RowBits)1));
            A &= x | (x * neg1);
        }
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r)
            A &= Z[r] | (Z[r] * neg1);
    }
    uint32_t M = 0xffffffffu;  // columns >= checkpoint
    for (;;) {
        if (A == 0u) {
            // a live row runs past the word end: remember the others
            RowBits d = deadbits;
#pragma unroll
            for (int r = 0; r < NR; ++r)
                d |= (RowBits)((Z[r] & M) != 0u) << r;
            deadbits = d;
            return;
        }
        deadbits = 0;  // an obstacle ends every run: fresh checkpoint
        const int e = base + ffs32(A) - 1;  // end of the escape segment
        if (e >= m) {                       // reached the destination
            finished = true;
            return;
        }
        ++count;                            // its obstacle
        if (count > E) {                    // delay exceeds E: reject
            finished = true;
            return;
        }
        const int c = e + 1;                // new checkpoint
        if (c >= base + 32)
            return;
        M = 0xffffffffu << (c - base);
        A = 0xffffffffu;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const uint32_t x = Z[r] & M;
            A &= x | (x * neg1);
        }
    }
}

// Route one pair of length m with threshold E (E == EMAX when EXACT);
// returns min(count, E+1).  Rows |s| > min(E, EMAX) are never built.
// neg1 must hold 0xffffffff: the subtractions are multiply-adds by values
// derived from it at run time, which issue on the FMA pipe and leave the
// busier ALU pipe to the logic ops.
template <int EMAX, bool EXACT, class Seq>
SS_HD int rw_route(const Seq &Qs, const Seq &Rs, int m, int E, uint32_t neg1)
{
    constexpr int NR = 2 * EMAX + 1;
    // bitmask of rows that met an obstacle since the checkpoint (crossing)
    using RowBits = typename std::conditional<(NR <= 32), uint32_t,
                                              uint64_t>::type;
    const int W32 = (m + 31) >> 5;
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
        // Eq. 1 case 4 on the columns below m: row s < 0 reads query
        // indices below 0 only in word 0, row s > 0 reads indices past m
        // only within 32 + s columns of m, and row 0 never leaves 0..m-1.
        const bool lo_edge = k == 0;
        const bool hi_edge = base + 32 + EMAX > m;
        // "Q base exists" plane around word k (bits of Q indices in 0..m-1),
        // shifted with each row like Q itself
        const uint32_t v_c = mask_below(m - base);
        const uint32_t v_n = mask_below(m - base - 32);
        // Eq. 1 for the 32 columns of word k, every row.  Columns past m are
        // not masked: whatever they hold can only place the longest run's end
        // at or beyond m, which is read as "reached the destination".
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
            if (!EXACT && (s > E || -s > E))
                z = 0xffffffffu;  // row outside this pair's 2E+1
            Z[r] = z;
        }
        // Greedy routing inside word k (checkpoint c <= base on entry).
        rw_word_smear<NR>(Z, deadbits, base, m, E, count, finished, neg1);
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
    uint32_t neg1;          // 0xffffffff (see rw_route)
    uint8_t *acc;
    int32_t *obs;
};

// Predicted routing cost of a staged pair: the fewest mismatches over its
// first 32 reference bases on the five central diagonals (s = -2..2),
// capped at 31.  Random pairs score high and are rejected early; similar
// pairs score low -- also those with an indel early on, which shift the
// main diagonal -- and route to the end.  (A cost model over the oracle's
// per-word iteration counts ranked 5 diagonals above 1, 3, 7 and 9, and
// above wider windows of bases.)  Words i of the pair are at sq[i * ld],
// sr[i * ld].
__device__ __forceinline__ int rw_cost_key(const uint32_t *sq,
                                           const uint32_t *sr, int ld,
                                           int w16)
{
    const uint32_t q0 = sq[0], q1 = w16 > 1 ? sq[ld] : 0u;
    const uint32_t q2 = w16 > 2 ? sq[2 * ld] : 0u;
    const uint32_t q3 = w16 > 3 ? sq[3 * ld] : 0u;
    const uint32_t r0 = sr[0], r1 = w16 > 1 ? sr[ld] : 0u;
    uint32_t qlo, qhi, qlo_n, qhi_n, rlo, rhi;
    planes_of(q0, q1, qlo, qhi);
    planes_of(q2, q3, qlo_n, qhi_n);
    planes_of(r0, r1, rlo, rhi);
    int k = __popc((qlo ^ rlo) | (qhi ^ rhi));
#pragma unroll
    for (int s = 1; s <= 2; ++s) {
        const uint32_t up = (funnel_r(qlo, qlo_n, s) ^ rlo) |
                            (funnel_r(qhi, qhi_n, s) ^ rhi);
        const uint32_t dn = (((qlo << s) ^ rlo) | ((qhi << s) ^ rhi)) &
                            (0xffffffffu << s);
        k = imin(k, imin(__popc(up), __popc(dn)));
    }
    return k < 31 ? k : 31;
}

// Counting sort of the tile's pairs by a cost key in 0..31 (thread t holds
// pair t's key, t < np): returns the pair this thread routes.  s_cnt must
// be zero on entry.
__device__ __forceinline__ int rw_sort_keys(int key, int np, int *s_cnt,
                                            uint8_t *s_perm)
{
    const int t = threadIdx.x;
    int rank = 0;
    if (t < np)
        rank = atomicAdd(&s_cnt[key], 1);
    __syncthreads();
    if (t < 32) {
        const int c = s_cnt[t];
        int x = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, off);
            if (t >= off)
                x += y;
        }
        s_cnt[t] = x - c;  // exclusive start of bucket t
    }
    __syncthreads();
    if (t < np)
        s_perm[s_cnt[key] + rank] = (uint8_t)t;
    __syncthreads();
    return s_perm[t];
}

// Order the tile's pairs by predicted cost (counting sort on the CTA):
// returns the pair this thread routes.  Word i of the tile's pair u is at
// sQ[u * pair_ld + i * word_ld] (likewise sR).  s_cnt must be zero on entry.
__device__ __forceinline__ int rw_sort_tile(const uint32_t *sQ,
                                            const uint32_t *sR, int pair_ld,
                                            int word_ld, int w16, int np,
                                            int *s_cnt, uint8_t *s_perm)
{
    const int t = threadIdx.x;
    const int key = t < np ? rw_cost_key(sQ + t * pair_ld, sR + t * pair_ld,
                                         word_ld, w16)
                           : 0;
    return rw_sort_keys(key, np, s_cnt, s_perm);
}

// The plain kernels walk the greedy one column at a time (rw_route_cols)
// from E = kRwColsMinE on, and at E = kRwColsMinE - 1 for reads of at most
// kRwColsShortM bases; row-wise (rw_route) below.  Measured on GB300 (10M
// pairs, edit rate U[0, 0.12]): at E = 5 row-wise 1.07 against 1.27 ms at
// 250 bp and 0.72 against 0.79 ms at 150 bp, but the walk 1.14 against
// 1.18 ms at 100 bp (30M pairs); from E = 6 the walk at every length.
constexpr int kRwColsMinE = 6;
constexpr int kRwColsShortM = 128;

// The plain kernels' routine for threshold E: min(count, E+1).
template <int E, class Seq>
__device__ __forceinline__ int rw_route_plain(const Seq &q, const Seq &r,
                                              int m, uint32_t neg1)
{
    if constexpr (E >= kRwColsMinE) {
        return rw_route_cols<E>(q, r, m, neg1);
    } else if constexpr (E == kRwColsMinE - 1) {
        if (m <= kRwColsShortM)
            return rw_route_cols<E>(q, r, m, neg1);
        return rw_route<E, true>(q, r, m, E, neg1);
    } else {
        return rw_route<E, true>(q, r, m, E, neg1);
    }
}

// Plain launch for long reads: uniform m and E, one thread per pair, one CTA
// per T pairs.  The CTA stages its pairs (128-bit loads when aligned), orders
// them by a predicted routing cost so that each warp holds pairs of similar
// cost (the warp then diverges less), routes them, and writes each result at
// the pair's own index.
template <int E>
__global__ void __launch_bounds__(128)
    k_rw_staged(const RwUniformArgs a)
{
    extern __shared__ uint32_t smem[];
    __shared__ int s_cnt[32];
    __shared__ uint8_t s_perm[128];
    const int T = blockDim.x;  // 128
    const int ld = T + 1;
    const int t = threadIdx.x;
    const int64_t p0 = (int64_t)blockIdx.x * T;
    const int64_t left = a.n - p0;
    const int np = left < T ? (int)left : T;
    uint32_t *sQ = smem;
    uint32_t *sR = smem + (size_t)a.w16 * ld;
    const int w16 = a.w16;
    const int total = np * w16;
    const uint32_t *gq = a.reads + p0 * w16;
    const uint32_t *gr = a.refs + p0 * w16;
    if (t < 32)
        s_cnt[t] = 0;
    // stage, transposed: packed word i of pair u at [i * ld + u]
    int done = 0;
    if (((((uintptr_t)gq) | ((uintptr_t)gr)) & 15) == 0) {
        const int nv = total >> 2;
        const uint4 *vq = reinterpret_cast<const uint4 *>(gq);
        const uint4 *vr = reinterpret_cast<const uint4 *>(gr);
        for (int v = t; v < nv; v += T) {
            const uint4 q = __ldg(vq + v), r = __ldg(vr + v);
            const uint32_t idx = (uint32_t)v * 4u;
            uint32_t u = fast_div(idx, (uint32_t)w16, a.w16_magic);
            uint32_t i = idx - u * (uint32_t)w16;
            const uint32_t qq[4] = {q.x, q.y, q.z, q.w};
            const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                sQ[i * ld + u] = qq[c];
                sR[i * ld + u] = rr[c];
                if (++i == (uint32_t)w16) {
                    i = 0;
                    ++u;
                }
            }
        }
        done = nv * 4;
    }
    for (int idx = done + t; idx < total; idx += T) {
        const uint32_t u = fast_div((uint32_t)idx, (uint32_t)w16,
                                    a.w16_magic);
        const uint32_t i = (uint32_t)idx - u * (uint32_t)w16;
        sQ[i * ld + u] = __ldg(gq + idx);
        sR[i * ld + u] = __ldg(gr + idx);
    }
    __syncthreads();
    // order the CTA's pairs by predicted cost
    const int u = rw_sort_tile(sQ, sR, 1, ld, w16, np, s_cnt, s_perm);
    if (t < np) {
        const SmemSeq q{sQ + u, ld, w16};
        const SmemSeq r{sR + u, ld, w16};
        const int cnt = rw_route_plain<E>(q, r, a.m, a.neg1);
        a.acc[p0 + u] = (uint8_t)(cnt <= E);
        a.obs[p0 + u] = cnt;
    }
}

constexpr int kRwGroup = 8;                  // tiles per CTA
constexpr int kRwPipeMaxW16 = 16;            // m <= 256
constexpr uint64_t kRwWaitNs = 2000000000ull;  // 2 s per stage wait

// Shared-memory stages of the pipelined kernel, a compile-time constant so
// that a tile's stage and barrier phase are bit operations.  Two stages: a
// third adds shared memory (fewer resident CTAs) and measured no faster;
// more tiles per CTA than 8 unbalance the CTAs' routing cost.
constexpr int kRwStages = 2;
constexpr int kRwPadWords = 4;  // read past the last pair of the ring
// Dynamic shared memory of the pipelined kernel for w16 words per sequence.
SS_HD size_t rw_pipe_smem(int w16)
{
    return ((size_t)kRwStages * 2u * kRwThreads * (size_t)w16 +
            kRwPadWords) * 4u;
}

struct RwPipeArgs {
    const uint32_t *reads;  // packed, pair p at word p * w16
    const uint32_t *refs;
    int64_t n;
    int64_t ntiles;         // ceil(n / kRwThreads)
    int32_t m;
    int32_t w16;
    int32_t bulk;           // inputs 16-byte aligned: full tiles bulk-copied
    int32_t group;          // tiles per CTA
    uint32_t neg1;          // 0xffffffff (see rw_route)
    uint8_t *acc;
    int32_t *obs;
    int *status;
};

// Arguments, grid and dynamic shared memory of a pipelined launch over n
// pairs of length m (w16 <= kRwPipeMaxW16); false if the grid would exceed
// 2^31 - 1 CTAs.
inline bool rw_pipe_config(const uint32_t *reads, const uint32_t *refs,
                           int64_t n, int32_t m, uint8_t *acc, int32_t *obs,
                           int *status, RwPipeArgs &a, unsigned &grid,
                           size_t &smem)
{
    const int w16 = (m + 15) / 16 > 1 ? (m + 15) / 16 : 1;
    a.reads = reads;
    a.refs = refs;
    a.n = n;
    a.ntiles = (n + kRwThreads - 1) / kRwThreads;
    a.m = m;
    a.w16 = w16;
    a.group = kRwGroup;
    a.bulk = ((((uintptr_t)reads) | ((uintptr_t)refs)) & 15) == 0;
    a.neg1 = 0xffffffffu;
    a.acc = acc;
    a.obs = obs;
    a.status = status;
    smem = rw_pipe_smem(w16);
    const int64_t groups = (a.ntiles + a.group - 1) / a.group;
    grid = (unsigned)groups;
    return groups <= 0x7fffffff;
}

// The pipelined tile loop of the uniform launches (m <= 256): CTA b takes
// tiles group * b .. group * b + group - 1 of kRwThreads pairs each into
// pair-major shared-memory stages filled by bulk copies, orders each tile by
// the predicted cost (SORT), and routes pair u of the tile with
// route(Q, R) -> min(count, E+1) over its staged words.  Reads past the
// pair land in the stage (Q is followed by the tile's R words); R may be
// read up to kRwPadWords words past.  Results go to the pair's own index.
template <bool SORT, class Route>
__device__ __forceinline__ void rw_pipe_run(const RwPipeArgs &a, int E,
                                            Route route)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ __align__(8) uint64_t full[kRwStages];
    __shared__ int s_cnt[32];
    __shared__ uint8_t s_perm[kRwThreads];
    const int t = threadIdx.x;
    const int w16 = a.w16;
    constexpr int S = kRwStages;
    const uint32_t tile_words = (uint32_t)kRwThreads * (uint32_t)w16;
    const uint32_t tile_bytes = tile_words * 4u;
    // tile j < group of this CTA is global tile group * blockIdx.x + j; it
    // is bulk-copied iff the inputs are aligned and the tile is full
    auto tile_of = [&](int64_t j) {
        return j < a.group ? (int64_t)blockIdx.x * a.group + j : a.ntiles;
    };
    auto by_copy = [&](int64_t tile) {
        return a.bulk && tile < a.ntiles &&
               (tile + 1) * (int64_t)kRwThreads <= a.n;
    };
    auto issue = [&](int s, int64_t tile) {
        uint32_t *dq = smem + (size_t)s * 2u * tile_words;
        mbar_arrive_expect_tx(&full[s], 2u * tile_bytes);
        bulk_load(dq, a.reads + tile * tile_words, tile_bytes, &full[s]);
        bulk_load(dq + tile_words, a.refs + tile * tile_words, tile_bytes,
                  &full[s]);
    };
    if (t == 0) {
        for (int s = 0; s < S; ++s)
            mbar_init(&full[s], 1);
        mbar_init_fence();
    }
    if (t < 32)
        s_cnt[t] = 0;
    __syncthreads();
    if (t == 0)
        for (int j = 0; j < S; ++j)
            if (by_copy(tile_of(j)))
                issue(j, tile_of(j));
    for (int j = 0;; ++j) {
        const int64_t tile = tile_of(j);
        if (tile >= a.ntiles)
            break;
        const int s = (int)((uint32_t)j % S);
        uint32_t *sQ = smem + (size_t)s * 2u * tile_words;
        uint32_t *sR = sQ + tile_words;
        const int64_t p0 = tile * kRwThreads;
        const int np = (int)min((int64_t)kRwThreads, a.n - p0);
        if (by_copy(tile)) {
            const bool ok = mbar_wait_bounded(
                &full[s], ((uint32_t)j / S) & 1u, kRwWaitNs);
            if (__syncthreads_or(!ok)) {
                if (t == 0) {
                    atomicOr(a.status, kStatusTimeout);
                    // drain the copies still in flight into this CTA
                    for (int k = j; k < j + S; ++k)
                        if (by_copy(tile_of(k)))
                            mbar_wait_bounded(&full[(uint32_t)k % S],
                                              ((uint32_t)k / S) & 1u,
                                              kRwWaitNs);
                }
                return;
            }
        } else {
            const uint32_t *gq = a.reads + p0 * w16;
            const uint32_t *gr = a.refs + p0 * w16;
            for (int idx = t; idx < np * w16; idx += kRwThreads) {
                sQ[idx] = __ldg(gq + idx);
                sR[idx] = __ldg(gr + idx);
            }
            __syncthreads();
        }
        int u = t;
        if (SORT)
            u = rw_sort_tile(sQ, sR, w16, 1, w16, np, s_cnt, s_perm);
        if (t < np) {
            const int cnt =
                route(SmemSeqPad{sQ + u * w16}, SmemSeqPad{sR + u * w16});
            a.acc[p0 + u] = (uint8_t)(cnt <= E);
            a.obs[p0 + u] = cnt;
        }
        if (SORT && t < 32)
            s_cnt[t] = 0;
        __syncthreads();  // stage s and the sort buffers are free again
        if (t == 0 && by_copy(tile_of(j + S)))
            issue(s, tile_of(j + S));
    }
}

// Plain launch: uniform m <= 256 and E, the exact greedy (row-wise below
// E = kRwColsMinE, the column walk from there); the cost sort from E = 2
// (below, nearly every pair routes in one or two steps).
template <int E>
__global__ void __launch_bounds__(128) k_rw_uniform(const RwPipeArgs a)
{
    rw_pipe_run<(E >= 2)>(a, E, [&](const SmemSeqPad &q,
                                    const SmemSeqPad &r) {
        return rw_route_plain<E>(q, r, a.m, a.neg1);
    });
}

}  // namespace ssk
