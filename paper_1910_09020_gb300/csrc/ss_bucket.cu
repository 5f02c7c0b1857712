// ss_bucket.cu -- K2 (bucketing) and the launch sequence of the bucketed,
// persistent form (K4) for mixed batches.
//
// One call = k_seg_direct (ss_seg.cu: input tiles of one length and
// threshold routed on the plain kernel's pipeline, the other tiles
// classified into a histogram and listed) -> scan -> scatter of the listed
// tiles' pairs (the permutation that groups them by class, longest first)
// -> one persistent kernel per class, each pulling work from its own atomic
// counter.  Nothing on this path synchronises with the host, so the whole
// sequence is captured once in a CUDA graph and replayed; in the graph each
// class kernel (and the scatter) sits in a conditional node that the scan
// kernel switches on only when its class has pairs, so a replay launches
// only the kernels with work.  Row-wise classes run on the caller's stream
// and column-wise classes on a second stream forked inside the graph, so
// the two families overlap.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "ss_bucket.cuh"
#include "ss_cw.cuh"
#include "ss_device.cuh"
#include "ss_internal.h"
#include "ss_rw.cuh"

namespace ssk {

// Conditional-node handles of a captured pass: one per class and one for
// the scatter; `on` is 0 outside a graph (nothing to switch).
struct ScanCond {
    cudaGraphConditionalHandle h[kClasses + 1];
    int on;
};

// Pass 2: exclusive scan of the histogram (one CTA of 1024 threads); in a
// graph, switches on the conditional node of every class that has pairs
// and that of the scatter if any pair was deferred to a class.
__global__ void __launch_bounds__(1024) k_scan(const BucketWs ws,
                                               const ScanCond c)
{
    __shared__ int part[1024];
    constexpr int per = (kKeys + 1023) / 1024;
    const int t = threadIdx.x;
    int local[per];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < per; ++i) {
        const int k = t * per + i;
        local[i] = k < kKeys ? ws.hist[k] : 0;
        sum += local[i];
    }
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // Hillis-Steele
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - sum;  // exclusive prefix of this thread's keys
#pragma unroll
    for (int i = 0; i < per; ++i) {
        const int k = t * per + i;
        if (k < kKeys) {
            ws.cursor[k] = run;
            if (k % kLenBins == 0)
                ws.ranges[2 * (k / kLenBins)] = run;
            if (k % kLenBins == kLenBins - 1)
                ws.ranges[2 * (k / kLenBins) + 1] = run + local[i];
        }
        run += local[i];
    }
    if (t < kClasses)
        ws.counters[t] = 0u;
    if (c.on) {
        __syncthreads();  // every class range written
        if (t < kClasses)
            cudaGraphSetConditional(c.h[t],
                                    ws.ranges[2 * t + 1] > ws.ranges[2 * t]);
        else if (t == kClasses)
            cudaGraphSetConditional(c.h[kClasses], part[1023] > 0);
    }
}

// Pass 3: scatter the pairs of the deferred tiles to their key ranges (one
// CTA per tile at a time; one atomic per distinct key per warp).
__global__ void __launch_bounds__(kRwThreads)
    k_scatter(const PairSet ps, const BucketWs ws, const TuneParams tp)
{
    const int nd = *ws.ndeferred;
    const int lane = threadIdx.x & 31;
    for (int d = blockIdx.x; d < nd; d += gridDim.x) {
        const int64_t p = (int64_t)ws.deferred[d] * kRwThreads + threadIdx.x;
        int key = -1;
        if (p < ps.n) {
            const int m = ps.len(p), E = ps.thr(p);
            const int cls = class_of_tuned(m, E, tp);
            if (cls >= 0)
                key = cls * kLenBins + len_bin_desc(m);
        }
        const unsigned act = __ballot_sync(0xffffffffu, key >= 0);
        if (key >= 0) {
            const unsigned same = __match_any_sync(act, key);
            const int leader = __ffs(same) - 1;
            int base = 0;
            if (lane == leader)
                base = atomicAdd(&ws.cursor[key], __popc(same));
            base = __shfl_sync(same, base, leader);
            ws.perm[base + __popc(same & ((1u << lane) - 1u))] = (int32_t)p;
        }
    }
}

// Serving: put the pairs of the CTA-per-pair classes that the long-pair
// queue takes into its ring (one thread per pair; an entry is published
// by its seq, written after the entry's other fields).  The batch's
// descriptor already holds how many there are (the host counts them with
// the same rule); a different count here latches kStatusUnsupported.
__global__ void __launch_bounds__(256)
    k_long_enqueue(const PairSet ps, const BucketWs ws, const LongHook h,
                   int expect, int *status)
{
    __shared__ int s_n;
    if (threadIdx.x == 0)
        s_n = 0;
    __syncthreads();
    int mine = 0;
    for (int cls = kRwClasses + kCwwClasses; cls < kClasses; ++cls) {
        const int begin = ws.ranges[2 * cls], end = ws.ranges[2 * cls + 1];
        for (int i = begin + (int)threadIdx.x; i < end; i += blockDim.x) {
            const int64_t p = ws.perm[i];
            const int m = ps.len(p);
            if (!long_queued(cls, m, eff_threshold(m, ps.thr(p))))
                continue;
            const unsigned long long pos = atomicAdd(h.q.tail, 1ull);
            LongEntry *e = h.q.ring + (pos & (kLongRing - 1));
            e->pair = p;
            e->batch = h.batch;
            __threadfence();
            atomicExch(&e->seq, (uint32_t)(pos + 1));
            ++mine;
        }
    }
    atomicAdd(&s_n, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_n != expect)
        atomicOr(status, kStatusUnsupported);
}

// Row-wise class: thread per pair, warps take 32 consecutive entries.
template <int EMAX>
__global__ void __launch_bounds__(128) k_rw_bucket(const CwArgs a)
{
    const int lane = threadIdx.x & 31;
    const int begin = a.ws.ranges[2 * a.cls];
    const int end = a.ws.ranges[2 * a.cls + 1];
    for (;;) {
        int base = 0;
        if (lane == 0)
            base = begin + (int)atomicAdd(&a.ws.counters[a.cls], 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= end)
            break;
        const int idx = base + lane;
        if (idx < end) {
            const int64_t p = a.ws.perm[idx];
            const int m = a.ps.len(p), E = a.ps.thr(p);
            const int64_t off = a.ps.off(p);
            const int w16 = (m + 15) >> 4;
            const GlobalSeq q{a.ps.reads + off, w16};
            const GlobalSeq r{a.ps.refs + off, w16};
            const int cnt = rw_route<EMAX, false>(q, r, m, E, a.neg1);
            a.ps.acc[p] = (uint8_t)(cnt <= E);
            a.ps.obs[p] = cnt;
        }
    }
}

// ---- host side -------------------------------------------------------------

size_t bucket_ws_bytes(int64_t n)
{
    const size_t keys = (size_t)kKeys * 4;
    const size_t tiles = (size_t)((n + kRwThreads - 1) / kRwThreads) * 4;
    return 2 * keys + 16 + (size_t)kClasses * 12 + 256 + tiles + 256 +
           (size_t)n * 4 + 256;
}

// Layout: hist and ndeferred first (cleared by one memset per pass), then
// cursors, class ranges, work counters, the deferred tiles and the
// permutation (each list 256-byte aligned).
BucketWs bucket_ws_at(void *base, int64_t n)
{
    char *p = (char *)base;
    BucketWs ws;
    ws.hist = (int *)p;
    p += (size_t)kKeys * 4;
    ws.ndeferred = (int *)p;
    p += 16;
    ws.cursor = (int *)p;
    p += (size_t)kKeys * 4;
    ws.ranges = (int *)p;
    p += (size_t)kClasses * 8;
    ws.counters = (unsigned *)p;
    p += (size_t)kClasses * 4;
    p = (char *)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    ws.deferred = (int32_t *)p;
    p += (size_t)((n + kRwThreads - 1) / kRwThreads) * 4;
    p = (char *)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    ws.perm = (int32_t *)p;
    return ws;
}

// Bytes cleared at the start of every pass (hist and ndeferred).
static size_t bucket_clear_bytes() { return (size_t)kKeys * 4 + 16; }

// Largest staged pair (in shared words) of each column-wise class.
int cw_class_slice_words(int cls)
{
    if (cls >= kRwClasses && cls < kRwClasses + kCwwClasses) {
        const int Mb = cww_mbound(cls - kRwClasses);
        return CwLayout::of(Mb, kCwwMaxE).words();
    }
    const int i = cls - kRwClasses - kCwwClasses;
    const int w = i / kCwcMbounds, b = i % kCwcMbounds;
    const int Mb = cwc_mbound(b);
    int Emax = w == kCwcWidths - 1 ? Mb - 1 : (32 * cwc_width(w) - 1) / 2;
    Emax = std::min(Emax, Mb - 1);
    return CwLayout::of(Mb, Emax).words();
}

namespace {

// Resident CTAs per SM of a kernel configuration (at least 1).
template <class KernelT>
int occupancy_per_sm(KernelT kernel, int threads, size_t smem)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads,
                                                      smem) != cudaSuccess ||
        per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    return per_sm;
}

// Resident CTAs per SM of every persistent kernel, computed once per device
// (outside any stream capture) together with the kernels' shared-memory
// attributes, which are per device; a launch over `sm_share` SMs uses
// per_sm * sm_share CTAs, so several bucketed passes can share the GPU side
// by side.  Written once under g_init_mu before `ready` is released; read
// only by threads that saw it set.
struct LaunchCfg {
    int rw[kRwClasses];
    int cw[3][kClasses];  // [subgrid 4/8/16][class]
    std::atomic<bool> ready{false};
};
LaunchCfg g_cfg[kMaxDevices];
std::mutex g_init_mu;

// The current device's configuration, or nullptr before bucket_init.
const LaunchCfg *launch_cfg()
{
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (d < 0 || d >= kMaxDevices ||
        !g_cfg[d].ready.load(std::memory_order_acquire))
        return nullptr;
    return &g_cfg[d];
}

int kidx(int k) { return k == 4 ? 0 : k == 16 ? 2 : 1; }

template <int K>
cudaError_t init_cw(LaunchCfg &cfg)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_cw_warp<K>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_cw_cta<K>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024)) != cudaSuccess)
        return e;
    for (int c = 0; c < kCwwClasses; ++c) {
        const int cls = kRwClasses + c;
        const size_t smem = (size_t)4 * cw_class_slice_words(cls) * 4;
        cfg.cw[kidx(K)][cls] = occupancy_per_sm(k_cw_warp<K>, 128, smem);
    }
    for (int w = 0; w < kCwcWidths; ++w)
        for (int b = 0; b < kCwcMbounds; ++b) {
            const int cls = cwc_class(w, b);
            const size_t smem = (size_t)cw_class_slice_words(cls) * 4;
            cfg.cw[kidx(K)][cls] =
                occupancy_per_sm(k_cw_cta<K>, cwc_width(w), smem);
        }
    return cudaSuccess;
}

}  // namespace

cudaError_t bucket_init()
{
    int d = -1;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess)
        return e;
    if (d < 0 || d >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_init_mu);
    LaunchCfg &cfg = g_cfg[d];
    if (cfg.ready.load(std::memory_order_relaxed))
        return cudaSuccess;
    if ((e = rw_init(d)) != cudaSuccess)
        return e;
    cfg.rw[0] = occupancy_per_sm(k_rw_bucket<1>, 128, 0);
    cfg.rw[1] = occupancy_per_sm(k_rw_bucket<3>, 128, 0);
    cfg.rw[2] = occupancy_per_sm(k_rw_bucket<7>, 128, 0);
    cfg.rw[3] = occupancy_per_sm(k_rw_bucket<15>, 128, 0);
    cfg.rw[4] = occupancy_per_sm(k_rw_bucket<31>, 128, 0);
    if ((e = init_cw<4>(cfg)) != cudaSuccess ||
        (e = init_cw<8>(cfg)) != cudaSuccess ||
        (e = init_cw<16>(cfg)) != cudaSuccess)
        return e;
    cfg.ready.store(true, std::memory_order_release);
    return cudaSuccess;
}

namespace {

// Whether captured class kernels sit in conditional (IF) nodes.
constexpr bool kCondNodes = true;

// Parallel branches of a captured pass: every kernel launched through
// launch_if while `on` depends only on the fork point (the nodes the
// capture stream depended on at fan_begin), and fan_end makes the stream
// depend on all of them, so the class kernels are independent graph
// branches whose launch latencies overlap.
struct Fan {
    bool on = false;
    std::vector<cudaGraphNode_t> fork, joined;
};

cudaError_t fan_begin(Fan &f, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    const cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr,
                                                   &deps, nullptr, &nd);
    if (e != cudaSuccess)
        return e;
    if (cs != cudaStreamCaptureStatusActive)
        return cudaErrorStreamCaptureInvalidated;
    f.fork.assign(deps, deps + nd);
    f.joined.clear();
    f.on = true;
    return cudaSuccess;
}

cudaError_t fan_end(Fan &f, cudaStream_t st)
{
    f.on = false;
    if (f.joined.empty())
        return cudaStreamUpdateCaptureDependencies(
            st, f.fork.data(), nullptr, f.fork.size(),
            cudaStreamSetCaptureDependencies);
    return cudaStreamUpdateCaptureDependencies(
        st, f.joined.data(), nullptr, f.joined.size(),
        cudaStreamSetCaptureDependencies);
}

// Launch `func` on `st`: directly, or -- while `st` is being captured with
// conditional handles (c.on) -- as the body of an IF node on handle h, so
// that the replayed graph runs it only when the scan switched h on.  With
// an active fan, the node is a new branch from the fork point.
template <class... Args>
cudaError_t launch_if(const ScanCond &c, Fan *fan, int h,
                      void (*func)(Args...), unsigned grid, unsigned block,
                      size_t smem, cudaStream_t st, Args... args)
{
    if (grid == 0)
        return cudaSuccess;
    cudaError_t e;
    if (fan && fan->on &&
        (e = cudaStreamUpdateCaptureDependencies(
             st, fan->fork.data(), nullptr, fan->fork.size(),
             cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return e;
    auto joined = [&]() -> cudaError_t {
        if (!fan || !fan->on)
            return cudaSuccess;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        const cudaError_t r = cudaStreamGetCaptureInfo(
            st, &cs, nullptr, nullptr, &deps, nullptr, &nd);
        if (r != cudaSuccess)
            return r;
        fan->joined.insert(fan->joined.end(), deps, deps + nd);
        return cudaSuccess;
    };
    if (!c.on) {
        func<<<grid, block, smem, st>>>(args...);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        return joined();
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr,
                                      &nd)) != cudaSuccess)
        return e;
    if (cs != cudaStreamCaptureStatusActive)
        return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = c.h[h];
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp)) !=
        cudaSuccess)
        return e;
    void *argv[] = {(void *)&args...};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.func = (void *)func;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = argv;
    cudaGraphNode_t kn = nullptr;
    if ((e = cudaGraphAddKernelNode(&kn, cp.conditional.phGraph_out[0],
                                    nullptr, 0, &kp)) != cudaSuccess)
        return e;
    if ((e = cudaStreamUpdateCaptureDependencies(
             st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return e;
    return joined();
}

// counts (may be null): an upper bound of each class's pairs known on the
// host; classes it bounds by 0 are not launched.
template <int K>
cudaError_t launch_cw_classes(const LaunchCfg &cfg, CwArgs a, int sm_share,
                              const ScanCond &c, Fan *fan, cudaStream_t st,
                              const int64_t *counts)
{
    cudaError_t e;
    for (int k = 0; k < kCwwClasses; ++k) {
        a.cls = kRwClasses + k;
        if (counts && counts[a.cls] == 0)
            continue;
        a.slice_words = cw_class_slice_words(a.cls);
        const size_t smem = (size_t)4 * a.slice_words * 4;
        if ((e = launch_if(c, fan, a.cls, k_cw_warp<K>,
                           (unsigned)(cfg.cw[kidx(K)][a.cls] * sm_share), 128,
                           smem, st, a)) != cudaSuccess)
            return e;
    }
    for (int w = 0; w < kCwcWidths; ++w)
        for (int b = 0; b < kCwcMbounds; ++b) {
            a.cls = cwc_class(w, b);
            if (counts && counts[a.cls] == 0)
                continue;
            a.slice_words = cw_class_slice_words(a.cls);
            const size_t smem = (size_t)a.slice_words * 4;
            if ((e = launch_if(c, fan, a.cls, k_cw_cta<K>,
                               (unsigned)(cfg.cw[kidx(K)][a.cls] * sm_share),
                               (unsigned)cwc_width(w), smem, st, a)) !=
                cudaSuccess)
                return e;
        }
    return cudaSuccess;
}

cudaError_t launch_rw_classes(const LaunchCfg &cfg, CwArgs a, int sm_share,
                              const ScanCond &c, Fan *fan, cudaStream_t st,
                              const int64_t *counts)
{
    void (*const kern[kRwClasses])(CwArgs) = {
        k_rw_bucket<rw_emax(0)>, k_rw_bucket<rw_emax(1)>,
        k_rw_bucket<rw_emax(2)>, k_rw_bucket<rw_emax(3)>,
        k_rw_bucket<rw_emax(4)>};
    for (int k = 0; k < kRwClasses; ++k) {
        a.cls = k;
        if (counts && counts[k] == 0)
            continue;
        const cudaError_t e =
            launch_if(c, fan, k, kern[k], (unsigned)(cfg.rw[k] * sm_share),
                      128, 0, st, a);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// The pass up to the class kernels: clear, direct tiles and
// classification, scan, scatter.  With c.on, the handles are created on
// the graph being captured on st first.
cudaError_t launch_front(const PairSet &ps, const BucketWs &ws,
                         const TuneParams &tp, int *status, int sm_count,
                         ScanCond &c, cudaStream_t st)
{
    cudaError_t e;
    if (c.on) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g)) !=
            cudaSuccess)
            return e;
        if (cs != cudaStreamCaptureStatusActive)
            return cudaErrorStreamCaptureInvalidated;
        for (int i = 0; i <= kClasses; ++i)
            if ((e = cudaGraphConditionalHandleCreate(
                     &c.h[i], g, 0, cudaGraphCondAssignDefault)) !=
                cudaSuccess)
                return e;
    }
    if ((e = cudaMemsetAsync(ws.hist, 0, bucket_clear_bytes(), st)) !=
        cudaSuccess)
        return e;
    SegArgs sa;
    sa.ps = ps;
    sa.ws = ws;
    sa.tp = tp;
    sa.ntiles = (ps.n + kRwThreads - 1) / kRwThreads;
    sa.neg1 = 0xffffffffu;
    sa.status = status;
    if ((e = launch_seg_direct(sa, st)) != cudaSuccess)
        return e;
    k_scan<<<1, 1024, 0, st>>>(ws, c);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    const int64_t want = sa.ntiles;
    const unsigned grid =
        (unsigned)std::min<int64_t>(want, (int64_t)sm_count * 8);
    return launch_if(c, nullptr, kClasses, k_scatter, grid, kRwThreads, 0, st,
                     ps, ws, tp);
}

}  // namespace

cudaError_t launch_bucketed(const PairSet &ps, const BucketWs &ws,
                            const TuneParams &tp, int *status, int sm_count,
                            cudaStream_t st, cudaStream_t side,
                            cudaEvent_t fork, cudaEvent_t join,
                            bool conditional, int *launches,
                            const LongHook *hook, int hook_expect,
                            const int64_t *class_counts)
{
    if (ps.n <= 0)
        return cudaSuccess;
    const LaunchCfg *cfg = launch_cfg();
    if (!cfg)
        return cudaErrorNotReady;
    cudaError_t e;
    ScanCond c;
    std::memset(&c, 0, sizeof c);
    c.on = conditional && kCondNodes ? 1 : 0;
    if ((e = launch_front(ps, ws, tp, status, sm_count, c, st)) !=
        cudaSuccess)
        return e;
    *launches += 3;
    const int sh = sm_count;  // persistent grids span this many SMs
    CwArgs a{ps, ws, 0, 0};
    if (hook) {
        // serving: the queue's share of the CTA-per-pair classes
        k_long_enqueue<<<1, 256, 0, st>>>(ps, ws, *hook, hook_expect, status);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        a.queued = 1;
        *launches += 1;
    }
    Fan fan;
    cudaStream_t cw_st = st;
    if (conditional) {
        // captured: every class kernel a branch from the scatter
        if ((e = fan_begin(fan, st)) != cudaSuccess)
            return e;
    } else {
        // direct: column-wise classes on the side stream
        if ((e = cudaEventRecord(fork, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess)
            return e;
        cw_st = side;
    }
    const int64_t *cc = class_counts;
    if ((e = launch_rw_classes(*cfg, a, sh, c, &fan, st, cc)) != cudaSuccess)
        return e;
    switch (tp.cw_subgrid) {
    case 4: e = launch_cw_classes<4>(*cfg, a, sh, c, &fan, cw_st, cc); break;
    case 16: e = launch_cw_classes<16>(*cfg, a, sh, c, &fan, cw_st, cc); break;
    default: e = launch_cw_classes<8>(*cfg, a, sh, c, &fan, cw_st, cc); break;
    }
    if (e != cudaSuccess)
        return e;
    *launches += kClasses + 1;
    if (conditional)
        return fan_end(fan, st);
    if ((e = cudaEventRecord(join, side)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

// The same kernel sequence on a single stream with direct launches, for
// callers that hold no context (no side stream, no events): used by the
// allocation-free entry point.
cudaError_t launch_bucketed_one_stream(const PairSet &ps, const BucketWs &ws,
                                       int *status, cudaStream_t st)
{
    if (ps.n <= 0)
        return cudaSuccess;
    const LaunchCfg *cfg = launch_cfg();
    if (!cfg)
        return cudaErrorNotReady;
    cudaError_t e;
    const TuneParams tp;
    int sm_count = 0, dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount,
                                    dev)) != cudaSuccess)
        return e;
    ScanCond c;
    std::memset(&c, 0, sizeof c);
    if ((e = launch_front(ps, ws, tp, status, sm_count, c, st)) !=
        cudaSuccess)
        return e;
    CwArgs a{ps, ws, 0, 0};
    if ((e = launch_rw_classes(*cfg, a, sm_count, c, nullptr, st,
                               nullptr)) != cudaSuccess)
        return e;
    return launch_cw_classes<8>(*cfg, a, sm_count, c, nullptr, st, nullptr);
}

}  // namespace ssk
