// ss_bucket.cu -- K2 (bucketing) and the launch sequence of the bucketed,
// persistent form (K4) for mixed batches.
//
// One call = classify + histogram -> scan -> scatter (the permutation that
// groups pairs by class, longest first) -> one persistent kernel per class,
// each pulling work from its own atomic counter.  Nothing on this path
// synchronises with the host, so the whole sequence is captured once in a
// CUDA graph and replayed.  Row-wise classes run on the caller's stream and
// column-wise classes on a second stream forked inside the graph, so the two
// families overlap.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>

#include "ss_bucket.cuh"
#include "ss_cw.cuh"
#include "ss_device.cuh"
#include "ss_internal.h"
#include "ss_rw.cuh"

namespace ssk {

constexpr int kBucketThreads = 256;

// Pass 1: class of every pair; pairs needing no routing (m == 0) or with
// invalid values are answered here.  Per-block histogram in shared memory.
__global__ void __launch_bounds__(kBucketThreads)
    k_classify(const PairSet ps, const BucketWs ws, const TuneParams tp,
               int *status)
{
    __shared__ int h[kKeys];
    for (int k = threadIdx.x; k < kKeys; k += blockDim.x)
        h[k] = 0;
    __syncthreads();
    int bad = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ps.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int m = ps.len(p), E = ps.thr(p);
        const int cls = class_of_tuned(m, E, tp);
        if (cls >= 0) {
            atomicAdd(&h[cls * kLenBins + len_bin_desc(m)], 1);
        } else if (cls == kClassNone) {
            ps.acc[p] = 1;
            ps.obs[p] = 0;
        } else {
            ps.acc[p] = 0;
            ps.obs[p] = -1;
            bad |= cls == kClassInvalid ? kStatusInvalidArg
                                        : kStatusUnsupported;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kKeys; k += blockDim.x)
        if (h[k])
            atomicAdd(&ws.hist[k], h[k]);
    if (bad)
        atomicOr(status, bad);
}

// Pass 2: exclusive scan of the histogram (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_scan(const BucketWs ws)
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
}

// Pass 3: scatter pair indices to their key ranges (same partition of pairs
// over blocks as pass 1; one global atomic per non-empty key per block).
__global__ void __launch_bounds__(kBucketThreads)
    k_scatter(const PairSet ps, const BucketWs ws, const TuneParams tp)
{
    __shared__ int h[kKeys];
    for (int k = threadIdx.x; k < kKeys; k += blockDim.x)
        h[k] = 0;
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ps.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int m = ps.len(p), E = ps.thr(p);
        const int cls = class_of_tuned(m, E, tp);
        if (cls >= 0)
            atomicAdd(&h[cls * kLenBins + len_bin_desc(m)], 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kKeys; k += blockDim.x)
        if (h[k])
            h[k] = atomicAdd(&ws.cursor[k], h[k]);  // block's base in perm
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ps.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int m = ps.len(p), E = ps.thr(p);
        const int cls = class_of_tuned(m, E, tp);
        if (cls >= 0) {
            const int pos = atomicAdd(&h[cls * kLenBins + len_bin_desc(m)], 1);
            ws.perm[pos] = (int32_t)p;
        }
    }
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
    return 2 * keys + (size_t)kClasses * 12 + (size_t)n * 4 + 1024;
}

BucketWs bucket_ws_at(void *base, int64_t n)
{
    char *p = (char *)base;
    BucketWs ws;
    ws.hist = (int *)p;
    p += (size_t)kKeys * 4;
    ws.cursor = (int *)p;
    p += (size_t)kKeys * 4;
    ws.ranges = (int *)p;
    p += (size_t)kClasses * 8;
    ws.counters = (unsigned *)p;
    p += (size_t)kClasses * 4;
    p = (char *)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    ws.perm = (int32_t *)p;
    (void)n;
    return ws;
}

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

template <int K>
cudaError_t launch_cw_classes(const LaunchCfg &cfg, CwArgs a, int sm_share,
                              cudaStream_t st)
{
    for (int c = 0; c < kCwwClasses; ++c) {
        a.cls = kRwClasses + c;
        a.slice_words = cw_class_slice_words(a.cls);
        const size_t smem = (size_t)4 * a.slice_words * 4;
        k_cw_warp<K><<<cfg.cw[kidx(K)][a.cls] * sm_share, 128, smem, st>>>(
            a);
    }
    for (int w = 0; w < kCwcWidths; ++w)
        for (int b = 0; b < kCwcMbounds; ++b) {
            a.cls = cwc_class(w, b);
            a.slice_words = cw_class_slice_words(a.cls);
            const size_t smem = (size_t)a.slice_words * 4;
            k_cw_cta<K><<<cfg.cw[kidx(K)][a.cls] * sm_share, cwc_width(w),
                          smem, st>>>(a);
        }
    return cudaGetLastError();
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

cudaError_t launch_bucketed(const PairSet &ps, const BucketWs &ws,
                            const TuneParams &tp, int *status, int sm_count,
                            cudaStream_t st, cudaStream_t side,
                            cudaEvent_t fork, cudaEvent_t join,
                            int *launches)
{
    if (ps.n <= 0)
        return cudaSuccess;
    cudaError_t e;
    const int64_t want = (ps.n + kBucketThreads - 1) / kBucketThreads;
    const int grid = (int)std::min<int64_t>(want, (int64_t)sm_count * 4);
    if ((e = cudaMemsetAsync(ws.hist, 0, (size_t)kKeys * 4, st)) !=
        cudaSuccess)
        return e;
    k_classify<<<grid, kBucketThreads, 0, st>>>(ps, ws, tp, status);
    k_scan<<<1, 1024, 0, st>>>(ws);
    k_scatter<<<grid, kBucketThreads, 0, st>>>(ps, ws, tp);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    *launches += 3;
    // fork: column-wise classes on the side stream
    if ((e = cudaEventRecord(fork, st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess)
        return e;
    const LaunchCfg *cfg = launch_cfg();
    if (!cfg)
        return cudaErrorNotReady;
    const int sh = sm_count;  // persistent grids span this many SMs
    CwArgs a{ps, ws, 0, 0};
    a.cls = 0;
    k_rw_bucket<1><<<cfg->rw[0] * sh, 128, 0, st>>>(a);
    a.cls = 1;
    k_rw_bucket<3><<<cfg->rw[1] * sh, 128, 0, st>>>(a);
    a.cls = 2;
    k_rw_bucket<7><<<cfg->rw[2] * sh, 128, 0, st>>>(a);
    a.cls = 3;
    k_rw_bucket<15><<<cfg->rw[3] * sh, 128, 0, st>>>(a);
    a.cls = 4;
    k_rw_bucket<31><<<cfg->rw[4] * sh, 128, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    switch (tp.cw_subgrid) {
    case 4: e = launch_cw_classes<4>(*cfg, a, sh, side); break;
    case 16: e = launch_cw_classes<16>(*cfg, a, sh, side); break;
    default: e = launch_cw_classes<8>(*cfg, a, sh, side); break;
    }
    if (e != cudaSuccess)
        return e;
    *launches += kRwClasses + kCwwClasses + kCwcWidths * kCwcMbounds;
    if ((e = cudaEventRecord(join, side)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

// The same kernel sequence on a single stream, for callers that hold no
// context (no side stream, no events): used by the allocation-free entry
// point.
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
    const int64_t want = (ps.n + kBucketThreads - 1) / kBucketThreads;
    const int grid = (int)std::min<int64_t>(want, (int64_t)sm_count * 4);
    if ((e = cudaMemsetAsync(ws.hist, 0, (size_t)kKeys * 4, st)) !=
        cudaSuccess)
        return e;
    k_classify<<<grid, kBucketThreads, 0, st>>>(ps, ws, tp, status);
    k_scan<<<1, 1024, 0, st>>>(ws);
    k_scatter<<<grid, kBucketThreads, 0, st>>>(ps, ws, tp);
    const int sh = sm_count;
    CwArgs a{ps, ws, 0, 0};
    a.cls = 0;
    k_rw_bucket<1><<<cfg->rw[0] * sh, 128, 0, st>>>(a);
    a.cls = 1;
    k_rw_bucket<3><<<cfg->rw[1] * sh, 128, 0, st>>>(a);
    a.cls = 2;
    k_rw_bucket<7><<<cfg->rw[2] * sh, 128, 0, st>>>(a);
    a.cls = 3;
    k_rw_bucket<15><<<cfg->rw[3] * sh, 128, 0, st>>>(a);
    a.cls = 4;
    k_rw_bucket<31><<<cfg->rw[4] * sh, 128, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    return launch_cw_classes<8>(*cfg, a, sh, st);
}

}  // namespace ssk
