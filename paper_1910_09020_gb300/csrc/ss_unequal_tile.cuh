// ss_unequal_tile.cuh -- the tile kernel for pairs of different lengths
// (ss_unequal.cu launches it; ss_unequal_x0.cu and ss_unequal_x1.cu hold
// its exact-threshold instantiations, split so that they compile in
// parallel).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "ss_internal.h"
#include "ss_rw.cuh"
#include "ss_unequal.cuh"

namespace ssk {

struct UnequalArgs {
    const uint32_t *reads;
    const int64_t *read_off;  // words
    const int32_t *read_len;  // bases
    const uint32_t *refs;
    const int64_t *ref_off;
    const int32_t *ref_len;
    const int32_t *E;         // per pair, or nullptr: e for all
    int32_t e;
    int64_t n;
    uint8_t *acc;
    int32_t *obs;
    int *status;
};

// How a pair is handled: answered or left to another class (0), or routed
// by this launch (1).
enum UqMode { kUqNone = 0, kUqRoute = 1 };
constexpr int kUqGroup = 1;  // tiles per CTA (A/B at 2M pairs: 1 ahead of 2, 4, 8)

// The words of a pair's first bases for the cost key (0 past its end).
__device__ __forceinline__ void uq_head(const uint32_t *g, int w16,
                                        uint32_t (&w)[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i)
        w[i] = i < w16 ? __ldg(g + i) : 0u;
}

// Thread per pair over tiles of kRwThreads consecutive pairs, kUqGroup
// tiles per CTA: each tile's pairs of this row class (rows in
// ELO+1..EMAX; with EXACT every pair's threshold is EMAX and the routine
// is the one for exactly that threshold) are ordered by the flank-aware cost key, so that a warp
// holds pairs of similar routing work, and each is routed from global
// memory by the thread the order assigns it to.  (Staging the pairs in
// shared memory first, gathered half a warp per pair, was slower: 0.17
// against 0.11 ms at E = 2 on 2M pairs, the gather's load latency exposed
// before every tile.)  With ELO < 0
// the launch also answers the pairs that need no routing and flags the
// invalid and unsupported ones.
template <int EMAX, int ELO, bool EXACT>
__global__ void __launch_bounds__(kRwThreads) k_unequal_tile(
    const UnequalArgs a)
{
    __shared__ int s_mq[kRwThreads], s_mr[kRwThreads], s_e[kRwThreads];
    __shared__ int64_t s_qo[kRwThreads], s_ro[kRwThreads];
    __shared__ uint8_t s_mode[kRwThreads];
    __shared__ int s_cnt[32];
    __shared__ uint8_t s_perm[kRwThreads];
    const int t = threadIdx.x;
    if (t < 32)
        s_cnt[t] = 0;
    // the counts zero before any thread of the tile adds to them
    __syncthreads();
    int bad = 0;
    const int64_t ntiles = (a.n + kRwThreads - 1) / kRwThreads;
    for (int j = 0; j < kUqGroup; ++j) {
        const int64_t tile = (int64_t)blockIdx.x * kUqGroup + j;
        if (tile >= ntiles)
            break;
        const int64_t p0 = tile * kRwThreads;
        const int np = (int)min((int64_t)kRwThreads, a.n - p0);
        const int64_t p = p0 + t;
        int mQ = 0, mR = 0, E = 0, mode = kUqNone, key = 31;
        int64_t qo = 0, ro = 0;
        if (t < np) {
            mQ = a.read_len[p];
            mR = a.ref_len[p];
            E = a.E ? a.E[p] : a.e;
            const int rows =
                (mQ < 0 || mR < 0 || E < 0) ? -2 : unequal_rows(mQ, mR, E);
            if (rows == -2) {
                if (ELO < 0) {
                    a.acc[p] = 0;
                    a.obs[p] = -1;
                    bad |= kStatusInvalidArg;
                }
            } else if (rows < 0) {
                if (ELO < 0) {
                    a.acc[p] = 1;
                    a.obs[p] = 0;
                }
            } else if (rows > kRwMaxE) {
                if (ELO < 0) {
                    a.acc[p] = 0;
                    a.obs[p] = -1;
                    bad |= kStatusUnsupported;
                }
            } else if (rows > ELO && rows <= EMAX) {
                mode = kUqRoute;
                qo = a.read_off[p];
                ro = a.ref_off[p];
                uint32_t wq[4], wr[4];
                uq_head(a.reads + qo, (mQ + 15) >> 4, wq);
                uq_head(a.refs + ro, (mR + 15) >> 4, wr);
                key = uq_cost_key(wq, wr, E);
            }
        }
        s_mq[t] = mQ;
        s_mr[t] = mR;
        s_e[t] = E;
        s_qo[t] = qo;
        s_ro[t] = ro;
        s_mode[t] = (uint8_t)mode;
        const int u = rw_sort_keys(key, np, s_cnt, s_perm);
        if (t < np && s_mode[u] == kUqRoute) {
            const int uq = s_mq[u], ur = s_mr[u], uE = s_e[u];
            const GlobalSeq q{a.reads + s_qo[u], (uq + 15) >> 4};
            const GlobalSeq r{a.refs + s_ro[u], (ur + 15) >> 4};
            int cnt;
            if constexpr (EXACT)
                cnt = unequal_route_exact<EMAX>(q, uq, r, ur, 0xffffffffu);
            else
                cnt = unequal_route<EMAX>(q, uq, r, ur, uE, 0xffffffffu);
            a.acc[p0 + u] = (uint8_t)(cnt <= uE);
            a.obs[p0 + u] = cnt;
        }
        if (t < 32)
            s_cnt[t] = 0;
        __syncthreads();  // metadata and the sort buffers are free
    }
    if (bad)
        atomicOr(a.status, bad);
}

// Grid of a launch over n pairs (0 when it would exceed 2^31 - 1 CTAs).
inline unsigned unequal_grid(int64_t n)
{
    const int64_t ntiles = (n + kRwThreads - 1) / kRwThreads;
    const int64_t groups = (ntiles + kUqGroup - 1) / kUqGroup;
    return groups > 0x7fffffff ? 0u : (unsigned)groups;
}

template <int LO, int... I>
cudaError_t unequal_exact_range(int e, const UnequalArgs &a, unsigned grid,
                                cudaStream_t st,
                                std::integer_sequence<int, I...>)
{
    cudaError_t r = cudaErrorInvalidValue;
    ((e == LO + I
          ? (k_unequal_tile<LO + I, -1, true><<<grid, kRwThreads, 0, st>>>(a),
             r = cudaGetLastError(), 0)
          : 0),
     ...);
    return r;
}

// Exact-threshold launches by translation unit: e in 0..15 and 16..31.
cudaError_t launch_unequal_exact_x0(int e, const UnequalArgs &a,
                                    unsigned grid, cudaStream_t st);
cudaError_t launch_unequal_exact_x1(int e, const UnequalArgs &a,
                                    unsigned grid, cudaStream_t st);

}  // namespace ssk
