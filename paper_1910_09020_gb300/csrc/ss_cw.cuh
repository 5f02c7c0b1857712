// ss_cw.cuh -- K4 for large thresholds: one warp or one CTA per pair, maze
// bit-parallel across the rows ("column-wise"), with a row-wise extension
// of the surviving runs.
//
// Method (Section 2.4): from checkpoint c the greedy needs
//     p* = max over the 2E+1 rows s of (first obstacle of row s at or after c)
// then counts one obstacle and moves to p* + 1, or stops when p* reaches the
// row end (no obstacle) or the count exceeds E.
//
// GB300 mapping: thread word w owns 32 consecutive rows, s = -E + 32w + b.
// Column j of those rows is one 32-bit word -- a window of the Q bit planes
// at bit j - E + 32w compared with the broadcast base R[j] -- so one funnel
// shift per plane and two logic ops update 32 rows per column (the maze of
// Eq. 1 evaluated column by column, lazily from the checkpoint).  Phase 1
// runs K columns ("maze subgrid width") from c, AND-ing the columns into the
// set S of rows with no obstacle yet; rows of a random diagonal die after a
// few columns.  If S is still non-empty after K columns, phase 2 extends each
// surviving row with 32-column word compares (row-wise) until its first
// obstacle.  The group max of the per-thread candidates is p*.
//
// Pair data is staged in shared memory as bit planes (lo, hi, and a "Q base
// exists" plane qv that is 0 outside 1..m), with E/32 + 2 guard words on
// each side of Q so every window read stays in bounds.
#pragma once
#include <cstdint>

#include "ss_bucket.cuh"
#include "ss_device.cuh"

namespace ssk {

// Shared-memory layout of one staged pair.
struct CwLayout {
    int W32;  // 32-column words
    int GW;   // guard words on each side of Q
    int QW;   // words per Q plane
    int RW;   // words per R plane
    __host__ __device__ static CwLayout of(int m, int Ee)
    {
        CwLayout L;
        L.W32 = (m + 31) >> 5;
        L.GW = ((Ee + 31) >> 5) + 2;
        L.QW = L.W32 + 2 * L.GW + 2;
        L.RW = L.W32 + 2;
        return L;
    }
    __host__ __device__ int words() const { return 3 * QW + 2 * RW; }
};

// Stage pair (gq, gr, m) into sm (layout L) with `nthreads` threads.
SS_HD void cw_stage(uint32_t *sm, const CwLayout &L, const uint32_t *gq,
                    const uint32_t *gr, int m, int t, int nthreads)
{
    uint32_t *qlo = sm, *qhi = sm + L.QW, *qv = sm + 2 * L.QW;
    uint32_t *rlo = sm + 3 * L.QW, *rhi = rlo + L.RW;
    const int w16 = (m + 15) >> 4;
    for (int k = t; k < L.QW; k += nthreads) {
        const int kk = k - L.GW;
        uint32_t lo = 0, hi = 0, v = 0;
        if (kk >= 0 && kk < L.W32) {
            const uint32_t p0 = ldg(gq + 2 * kk);
            const uint32_t p1 = 2 * kk + 1 < w16 ? ldg(gq + 2 * kk + 1) : 0u;
            planes_of(p0, p1, lo, hi);
            v = mask_below(m - 32 * kk);
        }
        qlo[k] = lo;
        qhi[k] = hi;
        qv[k] = v;
    }
    for (int k = t; k < L.RW; k += nthreads) {
        uint32_t lo = 0, hi = 0;
        if (k < L.W32) {
            const uint32_t p0 = ldg(gr + 2 * k);
            const uint32_t p1 = 2 * k + 1 < w16 ? ldg(gr + 2 * k + 1) : 0u;
            planes_of(p0, p1, lo, hi);
        }
        rlo[k] = lo;
        rhi[k] = hi;
    }
}

SS_HD uint32_t win(const uint32_t *p, int bit)
{
    const int i = bit >> 5;
    return funnel_r(p[i], p[i + 1], bit & 31);
}

// Candidate p (max first obstacle) of row word w from checkpoint c.
template <int K>
SS_HD int cw_word(const uint32_t *sm, const CwLayout &L, int m, int Ee,
                  int c, int w)
{
    const uint32_t *qlo = sm, *qhi = sm + L.QW, *qv = sm + 2 * L.QW;
    const uint32_t *rlo = sm + 3 * L.QW, *rhi = rlo + L.RW;
    const int nrows = 2 * Ee + 1;
    uint32_t S = mask_below(nrows - 32 * w);  // rows of this word that exist
    const int qpos = c - Ee + 32 * w + 32 * L.GW;
    // 64-column windows of the three Q planes for these 32 rows
    const uint32_t al = win(qlo, qpos), bl = win(qlo, qpos + 32);
    const uint32_t ah = win(qhi, qpos), bh = win(qhi, qpos + 32);
    const uint32_t av = win(qv, qpos), bv = win(qv, qpos + 32);
    const uint32_t rl = win(rlo, c), rh = win(rhi, c);  // R[c .. c+31]
    // Phase 1: K columns, 32 rows per word operation.
#pragma unroll
    for (int d = 0; d < K; ++d) {
        if (c + d >= m)
            return m;  // some row of this word reaches the row end
        const uint32_t ql = funnel_r(al, bl, d);
        const uint32_t qh = funnel_r(ah, bh, d);
        const uint32_t qe = funnel_r(av, bv, d);
        const uint32_t bl_ = 0u - ((rl >> d) & 1u);  // R[c+d] broadcast
        const uint32_t bh_ = 0u - ((rh >> d) & 1u);
        S &= qe & ~((ql ^ bl_) | (qh ^ bh_));
        if (S == 0u)
            return c + d;  // the last rows of this word die at column c+d
    }
    // Phase 2: extend each surviving row word-wise until its first obstacle.
    int cand = c + K;
    while (S) {
        const int b = ffs32(S) - 1;
        S &= S - 1u;
        int j = c + K;
        const int qb = qpos + b;  // Q bit of this row at column c
        for (;;) {
            const int qq = qb + (j - c);
            uint32_t x = (win(qlo, qq) ^ win(rlo, j)) |
                         (win(qhi, qq) ^ win(rhi, j)) | ~win(qv, qq);
            x |= mask_from(m - j);  // columns past the row end
            if (x) {
                const int first = j + ffs32(x) - 1;
                cand = imax(cand, imin(first, m));
                break;
            }
            j += 32;
        }
        if (cand >= m)
            return m;
    }
    return cand;
}

struct CwArgs {
    PairSet ps;
    BucketWs ws;
    int cls;
    int slice_words;  // shared words per staged pair
    uint32_t neg1 = 0xffffffffu;  // passed at run time (see rw_route)
    int queued = 0;   // skip the pairs the serving queue takes
};

__host__ __device__ inline bool long_queued(int cls, int m, int Ee)
{
    return cls >= kRwClasses + kCwwClasses &&
           CwLayout::of(m, Ee).words() <= kLongWords / kLongTeams;
}

// Barrier of a team of nt threads (whole warps) with its own named
// barrier bar (1..15); bar 0: the whole CTA.
__device__ __forceinline__ void team_sync(int bar, int nt)
{
    if (bar == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" : : "r"(bar), "r"(nt) : "memory");
}

// Route one pair with a team of nt threads (t: the thread's index in the
// team; any number of row words): the pair staged into smem, then the
// greedy of Section 2.4 with one team maximum per step (red: two 32-entry
// buffers, buf toggles between steps).  Returns min(count, E+1) (count
// itself is capped by the loop).
template <int K>
__device__ __forceinline__ int cw_team_route(uint32_t *smem, int (*red)[32],
                                             int &buf, const uint32_t *gq,
                                             const uint32_t *gr, int m, int E,
                                             int t, int nt, int bar)
{
    const int lane = t & 31, warp = t >> 5, nwarp = nt >> 5;
    const int Ee = eff_threshold(m, E);
    const CwLayout L = CwLayout::of(m, Ee);
    cw_stage(smem, L, gq, gr, m, t, nt);
    team_sync(bar, nt);
    const int nwords = (2 * Ee + 1 + 31) >> 5;
    int c = 0, count = 0;
    for (;;) {
        int cand = -1;
        for (int w = t; w < nwords; w += nt)
            cand = imax(cand, cw_word<K>(smem, L, m, Ee, c, w));
        cand = __reduce_max_sync(0xffffffffu, cand);
        if (lane == 0)
            red[buf][warp] = cand;
        team_sync(bar, nt);
        int v = lane < nwarp ? red[buf][lane] : -1;
        const int pstar = __reduce_max_sync(0xffffffffu, v);
        buf ^= 1;
        if (pstar >= m)
            break;
        ++count;
        if (count > E)
            break;
        c = pstar + 1;
    }
    return count;
}

// The same with the whole CTA as the team.
template <int K>
__device__ __forceinline__ int cw_cta_route(uint32_t *smem, int (*red)[32],
                                            int &buf, const uint32_t *gq,
                                            const uint32_t *gr, int m, int E)
{
    return cw_team_route<K>(smem, red, buf, gq, gr, m, E, threadIdx.x,
                            blockDim.x, 0);
}

// Warp per pair; blockDim.x / 32 warps, each with its own slice.
template <int K>
__global__ void __launch_bounds__(128) k_cw_warp(const CwArgs a)
{
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint32_t *sm = smem + (size_t)warp * a.slice_words;
    const int begin = a.ws.ranges[2 * a.cls];
    const int end = a.ws.ranges[2 * a.cls + 1];
    for (;;) {
        int idx = 0;
        if (lane == 0)
            idx = begin + (int)atomicAdd(&a.ws.counters[a.cls], 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= end)
            break;
        const int64_t p = a.ws.perm[idx];
        const int m = a.ps.len(p), E = a.ps.thr(p);
        const int Ee = eff_threshold(m, E);
        const CwLayout L = CwLayout::of(m, Ee);
        const int64_t off = a.ps.off(p);
        cw_stage(sm, L, a.ps.reads + off, a.ps.refs + off, m, lane, 32);
        __syncwarp();
        const int nwords = (2 * Ee + 1 + 31) >> 5;  // <= 32
        int c = 0, count = 0;
        for (;;) {
            const int cand = lane < nwords ? cw_word<K>(sm, L, m, Ee, c, lane)
                                           : -1;
            const int pstar = __reduce_max_sync(0xffffffffu, cand);
            if (pstar >= m)
                break;  // the net reached the destination
            ++count;
            if (count > E)
                break;
            c = pstar + 1;
        }
        if (lane == 0) {
            a.ps.acc[p] = (uint8_t)(count <= E);
            a.ps.obs[p] = count;
        }
        __syncwarp();
    }
}

// CTA per pair (blockDim.x threads, any number of row words).
template <int K>
__global__ void __launch_bounds__(1024) k_cw_cta(const CwArgs a)
{
    extern __shared__ uint32_t smem[];
    __shared__ int red[2][32];
    __shared__ int s_idx;
    const int t = threadIdx.x;
    const int begin = a.ws.ranges[2 * a.cls];
    const int end = a.ws.ranges[2 * a.cls + 1];
    int buf = 0;
    for (;;) {
        if (t == 0)
            s_idx = begin + (int)atomicAdd(&a.ws.counters[a.cls], 1u);
        __syncthreads();
        const int idx = s_idx;
        if (idx >= end)
            break;
        const int64_t p = a.ws.perm[idx];
        const int m = a.ps.len(p), E = a.ps.thr(p);
        if (a.queued && long_queued(a.cls, m, eff_threshold(m, E))) {
            __syncthreads();  // s_idx is reused
            continue;         // routed by the serving queue's worker
        }
        const int64_t off = a.ps.off(p);
        const int count = cw_cta_route<K>(smem, red, buf, a.ps.reads + off,
                                          a.ps.refs + off, m, E);
        if (t == 0) {
            a.ps.acc[p] = (uint8_t)(count <= E);
            a.ps.obs[p] = count;
        }
        __syncthreads();  // slice and s_idx are reused by the next pair
    }
}

}  // namespace ssk
