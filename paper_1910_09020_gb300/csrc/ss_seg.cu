// ss_seg.cu -- the first kernel of the bucketed form: input tiles that are
// plain batches in disguise go through the plain kernel's pipeline.
//
// A mixed batch often holds long runs of pairs that share their length and
// threshold and sit back to back in memory (a mapper's candidates for reads
// of one length, or two such batches concatenated).  k_seg_direct walks the
// input in tiles of 128 consecutive pairs, groups of kSegGroup tiles per
// CTA.  A tile whose pairs all have the same m <= 256 and E <= 31 and whose
// packed words are contiguous is routed here exactly as the plain launch
// routes it (Section 2.4 on the implicit maze): its words bulk-copied into a
// shared-memory stage, its pairs ordered by predicted cost, each routed by
// the plain kernels' routine for that E (a run-time dispatch over the 32
// compile-time forms, uniform across the tile).  Any other tile is
// classified here, pair by pair, into the class histogram of the bucketed
// classes and listed as deferred; the scan, the scatter and the per-class
// persistent kernels then handle only those pairs.
//
// Each tile's per-pair metadata (length, threshold, word offset: the 16
// bytes per pair the bucketed form must read) is loaded two tiles ahead of
// its routing, so its latency hides behind the routing of the tiles before
// it, and the tile's bulk copies are issued one tile ahead, as in the plain
// kernel.  Waits on the copies are bounded like the plain kernel's.
#include <cuda_runtime.h>

#include <cstdint>

#include "ss_bucket.cuh"
#include "ss_device.cuh"
#include "ss_internal.h"
#include "ss_rw.cuh"

namespace ssk {

namespace {

constexpr int kSegStages = 2;
constexpr int kSegStageWords = 2 * kRwThreads * kRwPipeMaxW16;

// The plain kernels' routine for a run-time threshold e in [LO, HI): a
// binary dispatch over the compile-time forms (five tests per pair).
template <int LO, int HI>
__device__ __forceinline__ int seg_route(int e, const SmemSeqPad &q,
                                         const SmemSeqPad &r, int m,
                                         uint32_t neg1)
{
    if constexpr (HI - LO == 1) {
        return rw_route_plain<LO>(q, r, m, neg1);
    } else {
        constexpr int MID = (LO + HI) / 2;
        if (e < MID)
            return seg_route<LO, MID>(e, q, r, m, neg1);
        return seg_route<MID, HI>(e, q, r, m, neg1);
    }
}

struct SegMeta {
    int m, e;
    int64_t off;
};

// How a tile is handled: deferred to the bucketed classes, or routed here
// from a stage filled by bulk copies or by plain loads.
enum SegMode { kSegDeferred = 0, kSegBulk = 1, kSegLoads = 2 };

struct SegTile {
    int64_t off;  // word offset of the tile's first pair
    int m, e, np, mode;
};

__device__ __forceinline__ int seg_w16(int m) { return (m + 15) >> 4; }

// Classify the pairs of a deferred tile into the class histogram (one
// atomic per distinct key per warp) and answer those that need no routing.
__device__ void seg_defer(const SegArgs &a, int64_t tile, int np)
{
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int64_t p = tile * kRwThreads + t;
    int key = -1, bad = 0;
    if (t < np) {
        const int m = a.ps.len(p), E = a.ps.thr(p);
        const int cls = class_of_tuned(m, E, a.tp);
        if (cls >= 0) {
            key = cls * kLenBins + len_bin_desc(m);
        } else if (cls == kClassNone) {
            a.ps.acc[p] = 1;
            a.ps.obs[p] = 0;
        } else {
            a.ps.acc[p] = 0;
            a.ps.obs[p] = -1;
            bad = cls == kClassInvalid ? kStatusInvalidArg
                                       : kStatusUnsupported;
        }
    }
    const unsigned act = __ballot_sync(0xffffffffu, key >= 0);
    if (key >= 0) {
        const unsigned same = __match_any_sync(act, key);
        if (lane == __ffs(same) - 1)
            atomicAdd(&a.ws.hist[key], __popc(same));
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && lane == 0)
        atomicOr(a.status, bad);
    if (t == 0)
        a.ws.deferred[atomicAdd(a.ws.ndeferred, 1)] = (int32_t)tile;
}

}  // namespace

size_t seg_smem_bytes()
{
    return ((size_t)kSegStages * kSegStageWords + kRwPadWords) * 4u;
}

__global__ void __launch_bounds__(kRwThreads) k_seg_direct(const SegArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ __align__(8) uint64_t full[kSegStages];
    __shared__ SegTile s_tile[kSegStages];
    __shared__ int s_cnt[32];
    __shared__ uint8_t s_perm[kRwThreads];
    const int t = threadIdx.x;
    const int64_t first = (int64_t)blockIdx.x * kSegGroup;
    const int ntl = (int)min((int64_t)kSegGroup, a.ntiles - first);

    // this thread's pair and the first pair of tile j of the group
    auto meta = [&](int j, SegMeta &own, SegMeta &fst) {
        const int64_t p0 = (first + j) * kRwThreads;
        const int64_t p = p0 + t;
        if (p < a.ps.n)
            own = SegMeta{a.ps.len(p), a.ps.thr(p), a.ps.off(p)};
        else
            own = SegMeta{0, 0, 0};
        fst = SegMeta{a.ps.len(p0), a.ps.thr(p0), a.ps.off(p0)};
    };
    // decide how tile j is handled (every thread, one barrier) and, for a
    // bulk tile, issue its copies into stage s
    auto decide = [&](int j, int s, const SegMeta &own, const SegMeta &fst) {
        const int64_t p0 = (first + j) * kRwThreads;
        const int np = (int)min((int64_t)kRwThreads, a.ps.n - p0);
        const bool shape_ok = fst.m >= 1 && fst.m <= 16 * kRwPipeMaxW16 &&
                              fst.e >= 0 && fst.e <= kRwMaxE;
        const int w16 = seg_w16(fst.m);
        const bool mine_ok =
            t >= np || (own.m == fst.m && own.e == fst.e &&
                        own.off == fst.off + (int64_t)t * w16);
        const bool uniform = __syncthreads_and(shape_ok && mine_ok);
        if (t == 0) {
            SegTile ti{fst.off, fst.m, fst.e, np, kSegDeferred};
            if (uniform) {
                const uint32_t *gq = a.ps.reads + fst.off;
                const uint32_t *gr = a.ps.refs + fst.off;
                const bool aligned =
                    ((((uintptr_t)gq) | ((uintptr_t)gr)) & 15) == 0;
                ti.mode = aligned && np == kRwThreads ? kSegBulk : kSegLoads;
                if (ti.mode == kSegBulk) {
                    const uint32_t words = (uint32_t)kRwThreads * w16;
                    uint32_t *dq = smem + (size_t)s * kSegStageWords;
                    mbar_arrive_expect_tx(&full[s], 8u * words);
                    bulk_load(dq, gq, 4u * words, &full[s]);
                    bulk_load(dq + words, gr, 4u * words, &full[s]);
                }
            }
            s_tile[s] = ti;
        }
    };

    if (t == 0) {
        for (int s = 0; s < kSegStages; ++s)
            mbar_init(&full[s], 1);
        mbar_init_fence();
    }
    if (t < 32)
        s_cnt[t] = 0;
    __syncthreads();
    // the first two tiles' metadata loaded together, then decided; the
    // third's in flight while the first is routed
    SegMeta own, fst, own1, fst1;
    if (ntl > 0)
        meta(0, own, fst);
    if (ntl > 1)
        meta(1, own1, fst1);
    if (ntl > 0)
        decide(0, 0, own, fst);
    if (ntl > 1)
        decide(1, 1, own1, fst1);
    if (kSegStages < ntl)
        meta(kSegStages, own, fst);  // two tiles ahead
    uint32_t phase[kSegStages] = {0u, 0u};
    for (int j = 0; j < ntl; ++j) {
        const int s = j & (kSegStages - 1);
        __syncthreads();  // s_tile[s] written
        const SegTile ti = s_tile[s];
        const int64_t tile = first + j;
        const int64_t p0 = tile * kRwThreads;
        if (ti.mode == kSegDeferred) {
            seg_defer(a, tile, ti.np);
        } else {
            const int w16 = seg_w16(ti.m);
            uint32_t *sQ = smem + (size_t)s * kSegStageWords;
            uint32_t *sR = sQ + kRwThreads * w16;
            if (ti.mode == kSegBulk) {
                const bool ok = mbar_wait_bounded(&full[s], phase[s] & 1u,
                                                  kRwWaitNs);
                phase[s] += 1u;
                if (__syncthreads_or(!ok)) {
                    if (t == 0) {
                        atomicOr(a.status, kStatusTimeout);
                        // drain the copies still in flight into this CTA:
                        // this stage's (if it gave up) and the other's
                        if (!ok)
                            mbar_wait_bounded(&full[s], (phase[s] - 1u) & 1u,
                                              kRwWaitNs);
                        const int o = s ^ 1;
                        if (j + 1 < ntl && s_tile[o].mode == kSegBulk)
                            mbar_wait_bounded(&full[o], phase[o] & 1u,
                                              kRwWaitNs);
                    }
                    return;
                }
            } else {
                const uint32_t *gq = a.ps.reads + ti.off;
                const uint32_t *gr = a.ps.refs + ti.off;
                for (int i = t; i < ti.np * w16; i += kRwThreads) {
                    sQ[i] = __ldg(gq + i);
                    sR[i] = __ldg(gr + i);
                }
                __syncthreads();
            }
            const bool sort = ti.e >= 2;
            int u = t;
            if (sort)
                u = rw_sort_tile(sQ, sR, w16, 1, w16, ti.np, s_cnt, s_perm);
            if (t < ti.np) {
                const int cnt =
                    seg_route<0, kRwMaxE + 1>(ti.e, SmemSeqPad{sQ + u * w16},
                                              SmemSeqPad{sR + u * w16}, ti.m,
                                              a.neg1);
                a.ps.acc[p0 + u] = (uint8_t)(cnt <= ti.e);
                a.ps.obs[p0 + u] = cnt;
            }
            if (sort && t < 32)
                s_cnt[t] = 0;
        }
        if (j + kSegStages < ntl) {
            // stage s is free once every thread is past this tile (the
            // barrier inside decide)
            decide(j + kSegStages, s, own, fst);
            if (j + kSegStages + 1 < ntl)
                meta(j + kSegStages + 1, own, fst);
        }
    }
}

cudaError_t launch_seg_direct(const SegArgs &a, cudaStream_t st)
{
    const int64_t groups = (a.ntiles + kSegGroup - 1) / kSegGroup;
    if (groups <= 0)
        return cudaSuccess;
    if (groups > 0x7fffffff)
        return cudaErrorInvalidValue;
    k_seg_direct<<<(unsigned)groups, kRwThreads, seg_smem_bytes(), st>>>(a);
    return cudaGetLastError();
}

}  // namespace ssk
