// ss_api.cu -- the C ABI of include/ss.h: context, argument checks, workspace,
// kernel dispatch, CUDA-graph cache and autotuner.  Every step of the filter
// runs in the CUDA kernels; this file only validates, allocates workspace and
// launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/ss.h"
#include "ss_bucket.cuh"
#include "ss_device.cuh"
#include "ss_internal.h"
#include "ss_rw_launch.cuh"

namespace {

// Everything a captured graph of the bucketed path depends on.
struct GraphKey {
    const void *reads, *refs, *offsets, *lengths, *E, *acc, *obs, *ws;
    int32_t m, e;
    int64_t n;
    int rw_max_e, cw_subgrid;
    bool operator==(const GraphKey &o) const
    {
        return std::memcmp(this, &o, sizeof(GraphKey)) == 0;
    }
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
    uint64_t last_use;
};

// A captured segmented call: its format and segment table.
struct SegGraph {
    int format;
    std::vector<ss_segment> segs;
    cudaGraphExec_t exec;
    uint64_t last_use;
};

// Independent launches of one call go round-robin to the caller's stream
// and kLanes - 1 streams of the context.
constexpr int kLanes = 4;

}  // namespace

struct ss_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;   // graph capture and internal work
    cudaStream_t side = nullptr;     // column-wise classes (forked)
    cudaStream_t hstream[2] = {nullptr, nullptr};  // ss_filter_host pipeline
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaStream_t lane[kLanes - 1] = {};   // independent launches (forked)
    cudaEvent_t lane_fork = nullptr;
    cudaEvent_t lane_done[kLanes - 1] = {};
    int *d_status = nullptr;         // [0] latched device errors, [1] the
                                     // value ss_sync last took from [0]
    size_t budget = 0;
    void *ws = nullptr;              // workspace: one growable device block
    size_t ws_bytes = 0;
    ssk::TuneParams tune;
    std::vector<GraphEntry> graphs;
    std::vector<SegGraph> seg_graphs;
    uint64_t tick = 0;
    ss_counters counters{};
};

namespace {

constexpr size_t kMaxGraphs = 16;

int cuda_fail(cudaError_t e)
{
    (void)cudaGetLastError();  // clear a non-sticky error
    return e == cudaErrorMemoryAllocation ? SS_ERR_OOM : SS_ERR_CUDA;
}

#define SS_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess)                                               \
            return cuda_fail(e_);                                            \
    } while (0)

#define SS_TRY(call)                                                         \
    do {                                                                     \
        int rc_ = (call);                                                    \
        if (rc_ != SS_OK)                                                    \
            return rc_;                                                      \
    } while (0)

// Make the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

void drop_graphs(ss_ctx *ctx)
{
    for (GraphEntry &g : ctx->graphs)
        cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
    for (SegGraph &g : ctx->seg_graphs)
        cudaGraphExecDestroy(g.exec);
    ctx->seg_graphs.clear();
}

// Grow the workspace to at least `bytes` (within the budget).
int ensure_workspace(ss_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes)
        return SS_OK;
    if (bytes > ctx->budget)
        return SS_ERR_OOM;
    if (ctx->ws) {
        // the old block may still be read by work on any caller stream
        SS_CUDA(cudaDeviceSynchronize());
        drop_graphs(ctx);
        SS_CUDA(cudaFree(ctx->ws));
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    SS_CUDA(cudaMalloc(&ctx->ws, bytes));
    ctx->ws_bytes = bytes;
    ctx->counters.workspace_bytes = (int64_t)bytes;
    return SS_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// NULL selects the CUDA default stream, as in other CUDA libraries (and as
// torch's default stream handle is 0).
cudaStream_t pick_stream(void *stream) { return (cudaStream_t)stream; }

// Launches that do not depend on one another, spread over the caller's
// stream and the context's lane streams: the CTAs of the next kernel fill
// the SMs that the previous one's last wave leaves idle, instead of the GPU
// draining between them.  Job i runs on lane i % kLanes (lane 0: the
// caller's stream); the destructor joins every lane used back into the
// caller's stream, so what follows on it sees all the jobs' results.
class Lanes {
  public:
    Lanes(ss_ctx *ctx, cudaStream_t st) : ctx_(ctx), st_(st) {}
    Lanes(const Lanes &) = delete;
    Lanes &operator=(const Lanes &) = delete;
    ~Lanes() { (void)join(); }

    // The stream of job `job`; the jobs are asked for in launch order.
    cudaError_t stream(int job, cudaStream_t &out)
    {
        const int l = job % kLanes;
        out = st_;
        cudaError_t e;
        if (!forked_) {
            // the fork point: on the caller's stream before the first job,
            // so that no lane waits for a job of lane 0
            if ((e = cudaEventRecord(ctx_->lane_fork, st_)) != cudaSuccess)
                return e;
            forked_ = true;
        }
        if (l == 0)
            return cudaSuccess;
        if (!(used_ & (1u << l))) {
            if ((e = cudaStreamWaitEvent(ctx_->lane[l - 1], ctx_->lane_fork,
                                         0)) != cudaSuccess)
                return e;
            used_ |= 1u << l;
        }
        out = ctx_->lane[l - 1];
        return cudaSuccess;
    }

    cudaError_t join()
    {
        cudaError_t first = cudaSuccess;
        for (int l = 1; l < kLanes; ++l) {
            if (!(used_ & (1u << l)))
                continue;
            cudaError_t e = cudaEventRecord(ctx_->lane_done[l - 1],
                                            ctx_->lane[l - 1]);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(st_, ctx_->lane_done[l - 1], 0);
            if (e != cudaSuccess && first == cudaSuccess)
                first = e;
        }
        used_ = 0;
        forked_ = false;
        return first;
    }

  private:
    ss_ctx *ctx_;
    cudaStream_t st_;
    unsigned used_ = 0;
    bool forked_ = false;
};

static_assert(SS_SLICED_MAX_E == ssk::kSlicedMaxE, "sliced limit");
static_assert(SS_PLAIN_MAX_E == ssk::kRwMaxE && SS_PLAIN_MAX_M == ssk::kRwMaxM,
              "the header states the plain launch's limits");

bool plain_ok(int32_t m, int32_t e)
{
    return e <= ssk::kRwMaxE && m <= ssk::kRwMaxM;
}

// The bucketed persistent form over packed pairs, as a replayed CUDA graph
// (or direct launches).  The workspace must already hold the bucket area at
// its start.
int run_bucketed(ss_ctx *ctx, const ssk::PairSet &ps, cudaStream_t st,
                 bool use_graph)
{
    ssk::BucketWs ws = ssk::bucket_ws_at(ctx->ws, ps.n);
    int launches = 0;
    if (!use_graph) {
        SS_CUDA(ssk::launch_bucketed(ps, ws, ctx->tune, ctx->d_status,
                                     ctx->sm_count, st, ctx->side, ctx->fork,
                                     ctx->join, false, &launches));
        ctx->counters.launches += launches;
        return SS_OK;
    }
    GraphKey key;
    std::memset(&key, 0, sizeof key);
    key.reads = ps.reads;
    key.refs = ps.refs;
    key.offsets = ps.offsets;
    key.lengths = ps.lengths;
    key.E = ps.Es;
    key.acc = ps.acc;
    key.obs = ps.obs;
    key.ws = ctx->ws;
    key.m = ps.m;
    key.e = ps.e;
    key.n = ps.n;
    key.rw_max_e = ctx->tune.rw_max_e;
    key.cw_subgrid = ctx->tune.cw_subgrid;
    for (GraphEntry &g : ctx->graphs)
        if (g.key == key) {
            g.last_use = ++ctx->tick;
            SS_CUDA(cudaGraphLaunch(g.exec, st));
            ctx->counters.graph_replays += 1;
            return SS_OK;
        }
    // capture on the context's own stream (the caller's may be the legacy
    // default stream, which cannot be captured), replay on the caller's
    cudaGraph_t graph = nullptr;
    SS_CUDA(cudaStreamBeginCapture(ctx->stream,
                                   cudaStreamCaptureModeThreadLocal));
    cudaError_t le = ssk::launch_bucketed(ps, ws, ctx->tune, ctx->d_status,
                                          ctx->sm_count, ctx->stream,
                                          ctx->side, ctx->fork, ctx->join,
                                          true, &launches);
    cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (graph)
            cudaGraphDestroy(graph);
        return cuda_fail(le != cudaSuccess ? le : ce);
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess)
        return cuda_fail(ie);
    if (ctx->graphs.size() >= kMaxGraphs) {
        auto lru = std::min_element(
            ctx->graphs.begin(), ctx->graphs.end(),
            [](const GraphEntry &a, const GraphEntry &b) {
                return a.last_use < b.last_use;
            });
        cudaGraphExecDestroy(lru->exec);
        ctx->graphs.erase(lru);
    }
    ctx->graphs.push_back(GraphEntry{key, exec, ++ctx->tick});
    ctx->counters.launches += launches;  // kernels per replay
    SS_CUDA(cudaGraphLaunch(exec, st));
    ctx->counters.graph_replays += 1;
    return SS_OK;
}

// Packed pairs: plain launch when m and E are uniform and the plain kernel
// covers them (unless the caller forces the bucketed form), else bucketed.
int filter_packed(ss_ctx *ctx, const ssk::PairSet &ps, int flags,
                  cudaStream_t st)
{
    const int mode = flags & 3;
    const bool uniform = !ps.offsets && !ps.lengths && !ps.Es;
    if (uniform && mode != SS_MODE_BUCKETED && plain_ok(ps.m, ps.e)) {
        SS_CUDA(ssk::launch_rw_uniform(ps.e, ps.reads, ps.refs, ps.n, ps.m,
                                       ps.acc, ps.obs, ctx->d_status, st));
        ctx->counters.launches += 1;
        return SS_OK;
    }
    if (mode == SS_MODE_PLAIN)
        return uniform ? SS_ERR_UNSUPPORTED : SS_ERR_INVALID_ARG;
    if (ps.n > INT32_MAX)
        return SS_ERR_UNSUPPORTED;
    return run_bucketed(ctx, ps, st, !(flags & SS_FLAG_NO_GRAPH));
}

ssk::PairSet make_pairs(const void *reads, const void *refs,
                        const int64_t *offsets, const int32_t *lengths,
                        int32_t m, const int32_t *E, int32_t e, int64_t n,
                        uint8_t *acc, int32_t *obs)
{
    ssk::PairSet ps;
    ps.reads = (const uint32_t *)reads;
    ps.refs = (const uint32_t *)refs;
    ps.offsets = offsets;
    ps.lengths = lengths;
    ps.Es = E;
    ps.m = m;
    ps.e = e;
    ps.stride = ((int64_t)m + 15) / 16;
    ps.n = n;
    ps.acc = acc;
    ps.obs = obs;
    return ps;
}

}  // namespace

namespace ssk {

namespace {
// Set once per device by rw_init (under bucket_init's lock).
std::atomic<bool> g_rw_ready[kMaxDevices];

bool rw_ready_here()
{
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return d >= 0 && d < kMaxDevices &&
           g_rw_ready[d].load(std::memory_order_acquire);
}
}  // namespace

cudaError_t rw_init(int device)
{
    if (device < 0 || device >= kMaxDevices)
        return cudaErrorInvalidDevice;
    if (g_rw_ready[device].load(std::memory_order_acquire))
        return cudaSuccess;
    cudaError_t e;
    if ((e = rw_init_e0()) != cudaSuccess ||
        (e = rw_init_e1()) != cudaSuccess ||
        (e = rw_init_e2()) != cudaSuccess ||
        (e = rw_init_e3()) != cudaSuccess)
        return e;
    g_rw_ready[device].store(true, std::memory_order_release);
    return cudaSuccess;
}

cudaError_t launch_rw_uniform(int E, const uint32_t *reads,
                              const uint32_t *refs, int64_t n, int32_t m,
                              uint8_t *acc, int32_t *obs, int *status,
                              cudaStream_t st)
{
    if (E < 0 || E > kRwMaxE || !rw_ready_here())
        return cudaErrorInvalidValue;
    RwLaunch L{};
    const int w16 = std::max((m + 15) / 16, 1);
    const int64_t ntiles = (n + kRwThreads - 1) / kRwThreads;
    if (w16 <= kRwPipeMaxW16) {
        L.pipe = true;
        if (!rw_pipe_config(reads, refs, n, m, acc, obs, status, L.pa,
                            L.grid, L.smem))
            return cudaErrorInvalidValue;
    } else {
        L.pipe = false;
        RwUniformArgs &a = L.sa;
        a.reads = reads;
        a.refs = refs;
        a.n = n;
        a.m = m;
        a.w16 = w16;
        a.w16_magic = div_magic((uint32_t)w16);
        a.neg1 = 0xffffffffu;
        a.acc = acc;
        a.obs = obs;
        L.smem = (size_t)2 * (size_t)w16 * (kRwThreads + 1) * 4;
        if (ntiles > 0x7fffffff)
            return cudaErrorInvalidValue;
        L.grid = (unsigned)ntiles;
    }
    if (L.grid == 0)
        return cudaSuccess;
    if (E <= 9)
        return launch_rw_uniform_e0(E, L, st);
    if (E <= 17)
        return launch_rw_uniform_e1(E, L, st);
    if (E <= 24)
        return launch_rw_uniform_e2(E, L, st);
    return launch_rw_uniform_e3(E, L, st);
}

}  // namespace ssk

extern "C" {

int ss_version(void) { return 400; }

const char *ss_strerror(int code)
{
    switch (code) {
    case SS_OK: return "ok";
    case SS_ERR_INVALID_ARG: return "invalid argument";
    case SS_ERR_INVALID_BASE: return "input byte is not A/C/G/T";
    case SS_ERR_OOM: return "workspace exceeds the budget or device memory";
    case SS_ERR_CUDA: return "CUDA runtime error";
    case SS_ERR_TIMEOUT: return "device-side wait timed out";
    case SS_ERR_BUSY: return "no free slot";
    case SS_ERR_UNSUPPORTED: return "shape not supported by this build";
    default: return "unknown status";
    }
}

int64_t ss_packed_words(int64_t m) { return m <= 0 ? 0 : (m + 15) / 16; }

int64_t ss_sliced_words(int64_t m, int64_t n)
{
    if (m <= 0 || n <= 0)
        return 0;
    return 8 * ((m + 3) / 4) * ((n + 31) / 32);
}

int ss_create(ss_ctx **out, int device, size_t workspace_bytes)
{
    if (!out)
        return SS_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        (void)cudaGetLastError();
        return SS_ERR_CUDA;
    }
    if (device < 0 || device >= ndev)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(device);
    if (!g.ok)
        return SS_ERR_CUDA;
    ss_ctx *ctx = new ss_ctx();
    ctx->device = device;
    ctx->budget = workspace_bytes ? workspace_bytes : ((size_t)1 << 30);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->hstream[0], cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->hstream[1], cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->lane_fork, cudaEventDisableTiming) !=
            cudaSuccess ||
        cudaMalloc(&ctx->d_status, 2 * sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, 2 * sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        ss_destroy(ctx);
        return SS_ERR_CUDA;
    }
    for (int l = 0; l < kLanes - 1; ++l)
        if (cudaStreamCreateWithFlags(&ctx->lane[l], cudaStreamNonBlocking) !=
                cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->lane_done[l],
                                     cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            ss_destroy(ctx);
            return SS_ERR_CUDA;
        }
    ctx->sm_count = prop.multiProcessorCount;
    if (ssk::bucket_init() != cudaSuccess) {
        (void)cudaGetLastError();
        ss_destroy(ctx);
        return SS_ERR_CUDA;
    }
    *out = ctx;
    return SS_OK;
}

int ss_destroy(ss_ctx *ctx)
{
    if (!ctx)
        return SS_OK;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    drop_graphs(ctx);
    for (cudaStream_t s : {ctx->stream, ctx->side, ctx->hstream[0],
                           ctx->hstream[1]})
        if (s)
            cudaStreamDestroy(s);
    if (ctx->fork)
        cudaEventDestroy(ctx->fork);
    if (ctx->join)
        cudaEventDestroy(ctx->join);
    for (int l = 0; l < kLanes - 1; ++l) {
        if (ctx->lane[l])
            cudaStreamDestroy(ctx->lane[l]);
        if (ctx->lane_done[l])
            cudaEventDestroy(ctx->lane_done[l]);
    }
    if (ctx->lane_fork)
        cudaEventDestroy(ctx->lane_fork);
    if (ctx->ws)
        cudaFree(ctx->ws);
    if (ctx->d_status)
        cudaFree(ctx->d_status);
    delete ctx;
    return SS_OK;
}

int ss_pack(ss_ctx *ctx, const uint8_t *ascii, const int64_t *offsets,
            const int32_t *lengths, int32_t m, int64_t n, uint32_t *packed,
            const int64_t *packed_offsets, void *stream)
{
    if (!ctx || n < 0)
        return SS_ERR_INVALID_ARG;
    if (n == 0)
        return SS_OK;
    if (!ascii || !packed)
        return SS_ERR_INVALID_ARG;
    const bool var = offsets || lengths || packed_offsets;
    if (var && !(offsets && lengths && packed_offsets))
        return SS_ERR_INVALID_ARG;
    if (!var && m < 0)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(stream);
    if (var)
        SS_CUDA(ssk::launch_pack_varlen(ascii, offsets, lengths, n, packed,
                                        packed_offsets, ctx->d_status,
                                        ctx->sm_count, st));
    else
        SS_CUDA(ssk::launch_pack_fixed(ascii, n, m, packed, ctx->d_status,
                                       st));
    ctx->counters.launches += 1;
    return SS_OK;
}

int ss_pack_sliced(ss_ctx *ctx, const uint8_t *ascii, int32_t m, int64_t n,
                   uint32_t *sliced, void *stream)
{
    if (!ctx || n < 0 || m < 0)
        return SS_ERR_INVALID_ARG;
    if (n == 0 || m == 0)
        return SS_OK;
    if (!ascii || !sliced || ((uintptr_t)sliced & 15))
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok)
        return SS_ERR_CUDA;
    SS_CUDA(ssk::launch_pack_sliced(ascii, n, m, sliced, ctx->d_status,
                                    pick_stream(stream)));
    ctx->counters.launches += 1;
    return SS_OK;
}

// The plain launch over SS_FMT_SLICED2 input (fixed stride, uniform m and
// e, validated by the caller).
static int filter_sliced(ss_ctx *ctx, const uint32_t *q, const uint32_t *r,
                         int32_t m, int32_t e, int64_t n, uint8_t *acc,
                         int32_t *obs, cudaStream_t st)
{
    SS_CUDA(ssk::launch_sliced(q, r, n, m, e, acc, obs, st));
    ctx->counters.launches += 1;
    return SS_OK;
}

extern "C++" {
// A threshold sweep over SS_FMT_SLICED2 input (every e_list[t] in
// 0..kSlicedMaxE, checked by the caller): the distinct thresholds up to
// kSlicedSetMaxE share one pass over the pairs when there are two or more
// of them (their walks cost less than the pass), every other threshold gets
// its own launch.  The launches are independent (each writes its own
// results): they go to the lanes, the costliest (largest threshold) first,
// the shared pass last.  acc(t), obs(t): where threshold t's results go.
template <class Acc, class Obs>
static int sweep_sliced(ss_ctx *ctx, const uint32_t *q, const uint32_t *r,
                        int32_t m, const int32_t *e_list, int n_e, int64_t n,
                        Acc acc, Obs obs, cudaStream_t st)
{
    constexpr int S = ssk::kSlicedSetMaxE + 1;
    int first[S];
    for (int e = 0; e < S; ++e)
        first[e] = -1;
    int shared = 0;
    for (int t = 0; t < n_e; ++t) {
        const int e = e_list[t];
        if (e < S && first[e] < 0) {
            first[e] = t;
            ++shared;
        }
    }
    std::vector<int> own;  // thresholds with a launch of their own
    for (int t = 0; t < n_e; ++t) {
        const int e = e_list[t];
        if (!(shared >= 2 && e < S && first[e] == t))
            own.push_back(t);
    }
    std::stable_sort(own.begin(), own.end(), [&](int a, int b) {
        return e_list[a] > e_list[b];
    });
    Lanes lanes(ctx, st);
    int job = 0;
    cudaStream_t ls;
    for (int t : own) {
        SS_CUDA(lanes.stream(job++, ls));
        SS_TRY(filter_sliced(ctx, q, r, m, e_list[t], n, acc(t), obs(t), ls));
    }
    if (shared >= 2) {
        unsigned mask = 0;
        uint8_t *pa[S];
        int32_t *po[S];
        int i = 0;
        for (int e = 0; e < S; ++e)
            if (first[e] >= 0) {
                mask |= 1u << e;
                pa[i] = acc(first[e]);
                po[i] = obs(first[e]);
                ++i;
            }
        SS_CUDA(lanes.stream(job++, ls));
        SS_CUDA(ssk::launch_sliced_set(q, r, n, m, mask, pa, po, ls));
        ctx->counters.launches += 1;
    }
    SS_CUDA(lanes.join());
    return SS_OK;
}
}  // extern "C++"

int ss_filter_sweep(ss_ctx *ctx, const void *reads, const void *refs,
                    int format, int32_t m, const int32_t *e_list, int n_e,
                    int64_t n, void *stream, uint8_t *out_accept,
                    int32_t *out_obstacles)
{
    if (!ctx || n < 0 || m < 0 || n_e < 0 || (n_e > 0 && !e_list))
        return SS_ERR_INVALID_ARG;
    if (format != SS_FMT_ASCII && format != SS_FMT_PACKED2 &&
        format != SS_FMT_SLICED2)
        return SS_ERR_INVALID_ARG;
    bool all_sliced = true;
    for (int t = 0; t < n_e; ++t) {
        if (e_list[t] < 0)
            return SS_ERR_INVALID_ARG;
        all_sliced &= e_list[t] <= ssk::kSlicedMaxE;
    }
    if (n == 0 || n_e == 0)
        return SS_OK;
    if (!reads || !refs || !out_accept || !out_obstacles)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok)
        return SS_ERR_CUDA;
    cudaStream_t st = pick_stream(stream);
    if (m == 0) {
        // nothing to route: every pair accepted with 0 obstacles
        SS_CUDA(cudaMemsetAsync(out_accept, 1, (size_t)n * n_e, st));
        SS_CUDA(cudaMemsetAsync(out_obstacles, 0, (size_t)n * n_e * 4, st));
        ctx->counters.pairs += n * n_e;
        return SS_OK;
    }
    auto acc_at = [&](int64_t p0) {
        return [=](int t) { return out_accept + (size_t)t * n + p0; };
    };
    auto obs_at = [&](int64_t p0) {
        return [=](int t) { return out_obstacles + (size_t)t * n + p0; };
    };
    if (format == SS_FMT_SLICED2) {
        if ((((uintptr_t)reads) | ((uintptr_t)refs)) & 15)
            return SS_ERR_INVALID_ARG;
        if (!all_sliced)
            return SS_ERR_UNSUPPORTED;
        ctx->counters.pairs += n * n_e;
        return sweep_sliced(ctx, (const uint32_t *)reads,
                            (const uint32_t *)refs, m, e_list, n_e, n,
                            acc_at(0), obs_at(0), st);
    }
    if (format == SS_FMT_ASCII && all_sliced) {
        // packed once per chunk (whole groups) to the sliced layout in the
        // workspace, every threshold over it
        const size_t seq = (size_t)((m + 3) / 4) + 1;
        if (ctx->budget <= 2048)
            return SS_ERR_OOM;
        int64_t chunk = (int64_t)((ctx->budget - 2048) / (2 * seq));
        if (chunk < n)
            chunk &= ~(int64_t)31;
        if (chunk < 1)
            return SS_ERR_OOM;
        chunk = std::min(chunk, n);
        const size_t seq_bytes =
            align_up((size_t)ss_sliced_words(m, chunk) * 4, 256);
        SS_TRY(ensure_workspace(ctx, 2 * seq_bytes));
        uint32_t *pq = (uint32_t *)ctx->ws;
        uint32_t *pr = (uint32_t *)((char *)ctx->ws + seq_bytes);
        for (int64_t p0 = 0; p0 < n; p0 += chunk) {
            const int64_t cn = std::min(chunk, n - p0);
            {
                // the two sides' packs side by side
                Lanes pk(ctx, st);
                cudaStream_t ls;
                SS_CUDA(pk.stream(0, ls));
                SS_CUDA(ssk::launch_pack_sliced(
                    (const uint8_t *)reads + p0 * (int64_t)m, cn, m, pq,
                    ctx->d_status, ls));
                SS_CUDA(pk.stream(1, ls));
                SS_CUDA(ssk::launch_pack_sliced(
                    (const uint8_t *)refs + p0 * (int64_t)m, cn, m, pr,
                    ctx->d_status, ls));
                SS_CUDA(pk.join());
            }
            ctx->counters.launches += 2;
            SS_TRY(sweep_sliced(ctx, pq, pr, m, e_list, n_e, cn, acc_at(p0),
                                obs_at(p0), st));
        }
        ctx->counters.pairs += n * n_e;
        return SS_OK;
    }
    // one fixed-stride filter per threshold
    for (int t = 0; t < n_e; ++t)
        SS_TRY(ss_filter_batch(ctx, reads, refs, format, nullptr, nullptr, m,
                               nullptr, e_list[t], n, SS_MODE_AUTO, stream,
                               out_accept + (size_t)t * n,
                               out_obstacles + (size_t)t * n));
    return SS_OK;
}

extern "C++" {
// One segment's launch in the pair-major packed format (the segment checked
// by the caller).
static int segment_launch(ss_ctx *ctx, const ss_segment &s, cudaStream_t st)
{
    if (s.m == 0) {
        // nothing to route: every pair accepted with 0 obstacles
        SS_CUDA(cudaMemsetAsync(s.out_accept, 1, (size_t)s.n, st));
        SS_CUDA(cudaMemsetAsync(s.out_obstacles, 0, (size_t)s.n * 4, st));
        return SS_OK;
    }
    SS_CUDA(ssk::launch_rw_uniform(s.e, (const uint32_t *)s.reads,
                                   (const uint32_t *)s.refs, s.n, s.m,
                                   s.out_accept, s.out_obstacles,
                                   ctx->d_status, st));
    ctx->counters.launches += 1;
    return SS_OK;
}

// The segments' launches, side by side on the lanes in the given order;
// over the sliced layout, segments of one threshold share a launch (up to
// kSlicedMaxSegments each, equal and different lengths apart), placed
// where the first of them stands.  Every segment's m_ref is its reference
// length (the caller's 0 already replaced by m).
static int segments_launch(ss_ctx *ctx, int format,
                           const std::vector<ss_segment> &segs,
                           cudaStream_t st)
{
    Lanes lanes(ctx, st);
    cudaStream_t ls;
    int job = 0;
    if (format != SS_FMT_SLICED2) {
        for (const ss_segment &sg : segs) {
            SS_CUDA(lanes.stream(job++, ls));
            SS_TRY(segment_launch(ctx, sg, ls));
        }
        SS_CUDA(lanes.join());
        return SS_OK;
    }
    std::vector<bool> done(segs.size(), false);
    for (size_t i = 0; i < segs.size(); ++i) {
        if (done[i])
            continue;
        ssk::SlicedSegment grp[ssk::kSlicedMaxSegments];
        int k = 0;
        const bool free_ends = segs[i].m_ref != segs[i].m;
        for (size_t j = i; j < segs.size() && k < ssk::kSlicedMaxSegments;
             ++j) {
            if (done[j] || segs[j].e != segs[i].e ||
                (segs[j].m_ref != segs[j].m) != free_ends)
                continue;
            const ss_segment &sg = segs[j];
            grp[k++] = ssk::SlicedSegment{
                (const uint32_t *)sg.reads, (const uint32_t *)sg.refs, sg.n,
                sg.m, sg.out_accept, sg.out_obstacles, sg.m_ref};
            done[j] = true;
        }
        SS_CUDA(lanes.stream(job++, ls));
        SS_CUDA(free_ends
                    ? ssk::launch_sliced_free_segments(grp, k, segs[i].e, ls)
                    : ssk::launch_sliced_segments(grp, k, segs[i].e, ls));
        ctx->counters.launches += 1;
    }
    SS_CUDA(lanes.join());
    return SS_OK;
}

// A segment's time, roughly: the larger of its bytes at the HBM rate and
// its walk's logic operations (m_ref (6e + 3) / 32 per pair: one column
// per reference base) at the logic-pipe rate, in units where the two rates
// are 6.8 and 20 per unit time.
static double segment_cost(const ss_segment &s)
{
    const double bytes = (s.m + 3) / 4 + (s.m_ref + 3) / 4 + 5.0;
    const double ops = (double)s.m_ref * (6.0 * s.e + 3.0) / 32.0;
    return (double)s.n * std::max(bytes / 6.8, ops / 20.0);
}
}  // extern "C++"

int ss_filter_segments(ss_ctx *ctx, const ss_segment *segs, int n_seg,
                       int format, int flags, void *stream)
{
    if (!ctx || n_seg < 0 || (n_seg > 0 && !segs))
        return SS_ERR_INVALID_ARG;
    if (format != SS_FMT_SLICED2 && format != SS_FMT_PACKED2)
        return SS_ERR_INVALID_ARG;
    if (flags & ~SS_FLAG_NO_GRAPH)
        return SS_ERR_INVALID_ARG;
    std::vector<ss_segment> work;
    int64_t pairs = 0;
    bool unsupported = false;
    for (int i = 0; i < n_seg; ++i) {
        const ss_segment &s = segs[i];
        if (s.n < 0 || s.m < 0 || s.e < 0 || s.m_ref < 0)
            return SS_ERR_INVALID_ARG;
        if (s.n == 0)
            continue;
        if (!s.reads || !s.refs || !s.out_accept || !s.out_obstacles)
            return SS_ERR_INVALID_ARG;
        // the fields alone (the key of the graph cache compares bytes)
        ss_segment w;
        std::memset(&w, 0, sizeof w);
        w.reads = s.reads;
        w.refs = s.refs;
        w.n = s.n;
        w.m = s.m;
        w.e = s.e;
        w.out_accept = s.out_accept;
        w.out_obstacles = s.out_obstacles;
        w.m_ref = s.m_ref ? s.m_ref : s.m;
        if (format == SS_FMT_SLICED2) {
            if ((((uintptr_t)s.reads) | ((uintptr_t)s.refs)) & 15)
                return SS_ERR_INVALID_ARG;
            unsupported |= s.e > ssk::kSlicedMaxE;
        } else {
            unsupported |= w.m_ref != w.m || (s.m > 0 && !plain_ok(s.m, s.e));
        }
        work.push_back(w);
        pairs += s.n;
    }
    if (unsupported)
        return SS_ERR_UNSUPPORTED;
    if (work.empty())
        return SS_OK;
    std::stable_sort(work.begin(), work.end(),
                     [](const ss_segment &a, const ss_segment &b) {
                         return segment_cost(a) > segment_cost(b);
                     });
    DeviceGuard g(ctx->device);
    if (!g.ok)
        return SS_ERR_CUDA;
    cudaStream_t st = pick_stream(stream);
    ctx->counters.pairs += pairs;
    if (flags & SS_FLAG_NO_GRAPH)
        return segments_launch(ctx, format, work, st);
    const size_t key_bytes = work.size() * sizeof(ss_segment);
    for (SegGraph &sg : ctx->seg_graphs)
        if (sg.format == format && sg.segs.size() == work.size() &&
            std::memcmp(sg.segs.data(), work.data(), key_bytes) == 0) {
            sg.last_use = ++ctx->tick;
            SS_CUDA(cudaGraphLaunch(sg.exec, st));
            ctx->counters.graph_replays += 1;
            return SS_OK;
        }
    // capture on the context's own stream (the caller's may be the legacy
    // default stream, which cannot be captured), replay on the caller's
    cudaGraph_t graph = nullptr;
    SS_CUDA(cudaStreamBeginCapture(ctx->stream,
                                   cudaStreamCaptureModeThreadLocal));
    const int rc = segments_launch(ctx, format, work, ctx->stream);
    cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
    if (rc != SS_OK || ce != cudaSuccess) {
        if (graph)
            cudaGraphDestroy(graph);
        return rc != SS_OK ? rc : cuda_fail(ce);
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess)
        return cuda_fail(ie);
    if (ctx->seg_graphs.size() >= kMaxGraphs) {
        auto lru = std::min_element(
            ctx->seg_graphs.begin(), ctx->seg_graphs.end(),
            [](const SegGraph &a, const SegGraph &b) {
                return a.last_use < b.last_use;
            });
        cudaGraphExecDestroy(lru->exec);
        ctx->seg_graphs.erase(lru);
    }
    ctx->seg_graphs.push_back(SegGraph{format, work, exec, ++ctx->tick});
    SS_CUDA(cudaGraphLaunch(exec, st));
    ctx->counters.graph_replays += 1;
    return SS_OK;
}

int ss_filter_batch(ss_ctx *ctx, const void *reads, const void *refs,
                    int format, const int64_t *offsets,
                    const int32_t *lengths, int32_t m, const int32_t *E,
                    int32_t e, int64_t n, int flags, void *stream,
                    uint8_t *out_accept, int32_t *out_obstacles)
{
    if (!ctx || n < 0)
        return SS_ERR_INVALID_ARG;
    if (format != SS_FMT_ASCII && format != SS_FMT_PACKED2 &&
        format != SS_FMT_SLICED2)
        return SS_ERR_INVALID_ARG;
    if ((flags & 3) == 3)
        return SS_ERR_INVALID_ARG;
    if (n == 0)
        return SS_OK;
    if (!reads || !refs || !out_accept || !out_obstacles)
        return SS_ERR_INVALID_ARG;
    if (offsets && !lengths)
        return SS_ERR_INVALID_ARG;
    if ((!lengths && m < 0) || (!E && e < 0))
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok)
        return SS_ERR_CUDA;
    cudaStream_t st = pick_stream(stream);
    ctx->counters.pairs += n;

    const bool uniform_len = !offsets && !lengths;
    if (uniform_len && m == 0) {
        // nothing to route: every pair accepted with 0 obstacles
        SS_CUDA(cudaMemsetAsync(out_accept, 1, (size_t)n, st));
        SS_CUDA(cudaMemsetAsync(out_obstacles, 0, (size_t)n * 4, st));
        return SS_OK;
    }
    if (format == SS_FMT_SLICED2) {
        if (!uniform_len || E)
            return SS_ERR_INVALID_ARG;  // the layout has a fixed stride
        if ((((uintptr_t)reads) | ((uintptr_t)refs)) & 15)
            return SS_ERR_INVALID_ARG;
        if (e > ssk::kSlicedMaxE || (flags & 3) == SS_MODE_BUCKETED)
            return SS_ERR_UNSUPPORTED;
        return filter_sliced(ctx, (const uint32_t *)reads,
                             (const uint32_t *)refs, m, e, n, out_accept,
                             out_obstacles, st);
    }
    const bool needs_bucket = !(uniform_len && !E && plain_ok(m, e)) ||
                              (flags & 3) == SS_MODE_BUCKETED;
    if (format == SS_FMT_PACKED2) {
        if (needs_bucket)
            SS_TRY(ensure_workspace(ctx, ssk::bucket_ws_bytes(n)));
        return filter_packed(ctx,
                             make_pairs(reads, refs, offsets, lengths, m, E, e,
                                        n, out_accept, out_obstacles),
                             flags, st);
    }
    // ASCII input: fixed stride only; packed chunk by chunk into workspace.
    if (!uniform_len)
        return SS_ERR_UNSUPPORTED;  // pack first with ss_pack
    // a uniform threshold from 1 to kSlicedMaxE: packed to the bit-sliced
    // layout and filtered 32 pairs per thread (at E = 0 the pair-major
    // pack and filter are cheaper)
    const bool sliced = !E && e >= 1 && e <= ssk::kSlicedMaxE &&
                        (flags & 3) != SS_MODE_BUCKETED;
    const int64_t w16 = (m + 15) / 16;
    // bytes of one packed sequence (the sliced layout: 32 ceil(m/4) bytes
    // per group of 32 sequences)
    const size_t seq = sliced ? (size_t)((m + 3) / 4) + 1 : (size_t)w16 * 4;
    const size_t per_pair = 2 * seq + (needs_bucket ? 4 : 0);
    const size_t fixed =
        needs_bucket ? ssk::bucket_ws_bytes(0) + 2048 : 2048;
    if (ctx->budget <= fixed)
        return SS_ERR_OOM;
    int64_t chunk = (int64_t)((ctx->budget - fixed) / per_pair);
    if (sliced && chunk < n)
        chunk &= ~(int64_t)31;  // whole groups of 32 pairs
    if (chunk < 1)
        return SS_ERR_OOM;
    chunk = std::min(chunk, n);
    const size_t bws =
        needs_bucket ? align_up(ssk::bucket_ws_bytes(chunk), 256) : 0;
    const size_t seq_bytes =
        sliced ? align_up((size_t)ss_sliced_words(m, chunk) * 4, 256)
               : align_up((size_t)chunk * w16 * 4, 256);
    SS_TRY(ensure_workspace(ctx, bws + 2 * seq_bytes));
    uint32_t *pq = (uint32_t *)((char *)ctx->ws + bws);
    uint32_t *pr = (uint32_t *)((char *)ctx->ws + bws + seq_bytes);
    for (int64_t p0 = 0; p0 < n; p0 += chunk) {
        const int64_t cn = std::min(chunk, n - p0);
        const uint8_t *rq = (const uint8_t *)reads + p0 * (int64_t)m;
        const uint8_t *rr = (const uint8_t *)refs + p0 * (int64_t)m;
        if (sliced) {
            SS_CUDA(ssk::launch_pack_sliced(rq, cn, m, pq, ctx->d_status, st));
            SS_CUDA(ssk::launch_pack_sliced(rr, cn, m, pr, ctx->d_status, st));
            ctx->counters.launches += 2;
            SS_TRY(filter_sliced(ctx, pq, pr, m, e, cn, out_accept + p0,
                                 out_obstacles + p0, st));
            continue;
        }
        SS_CUDA(ssk::launch_pack_fixed(rq, cn, m, pq, ctx->d_status, st));
        SS_CUDA(ssk::launch_pack_fixed(rr, cn, m, pr, ctx->d_status, st));
        ctx->counters.launches += 2;
        const int32_t *Ec = E ? E + p0 : nullptr;
        SS_TRY(filter_packed(ctx,
                             make_pairs(pq, pr, nullptr, nullptr, m, Ec, e, cn,
                                        out_accept + p0, out_obstacles + p0),
                             flags | SS_FLAG_NO_GRAPH, st));
    }
    return SS_OK;
}

int ss_filter_host(ss_ctx *ctx, const void *reads, const void *refs,
                   int format, int32_t m, const int32_t *e_list, int n_e,
                   int64_t n, uint8_t *out_accept, int32_t *out_obstacles)
{
    if (!ctx || n < 0 || m < 0 || n_e < 0 || (n_e > 0 && !e_list))
        return SS_ERR_INVALID_ARG;
    if (format != SS_FMT_ASCII && format != SS_FMT_PACKED2)
        return SS_ERR_INVALID_ARG;
    bool all_plain = true;
    for (int t = 0; t < n_e; ++t) {
        if (e_list[t] < 0)
            return SS_ERR_INVALID_ARG;
        all_plain &= plain_ok(m, e_list[t]);
    }
    if (n == 0 || n_e == 0)
        return SS_OK;
    if (!reads || !refs || !out_accept || !out_obstacles)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok)
        return SS_ERR_CUDA;
    const int64_t w16 = (m + 15) / 16;
    // ASCII input with every threshold up to kSlicedMaxE: each chunk packed
    // once to the bit-sliced layout, every threshold filtered over it
    bool sliced = format == SS_FMT_ASCII && m > 0;
    for (int t = 0; t < n_e; ++t)
        sliced &= e_list[t] <= ssk::kSlicedMaxE;
    // bytes of one sequence in the input format
    const size_t seq_in = format == SS_FMT_ASCII ? (size_t)m : (size_t)w16 * 4;
    const size_t packed = sliced ? (size_t)((m + 3) / 4) + 1
                                 : (size_t)w16 * 4;
    const size_t per_pair = 2 * seq_in +
                            (format == SS_FMT_ASCII ? 2 * packed : 0) +
                            (size_t)n_e * 5 + (all_plain ? 0 : 2);
    // two pipeline slots, each holding one chunk.  The copies in bound the
    // pipeline (the host link is slower than the filter), so the time not
    // overlapped is the first chunk's copy and the last chunk's compute and
    // copy back: chunks of 2M pairs keep both short and each launch still
    // fills the GPU.
    int64_t chunk = (int64_t)(ctx->budget / (2 * per_pair + 2048));
    chunk = std::min<int64_t>(chunk, (int64_t)1 << 21);
    if (sliced && chunk < n)
        chunk &= ~(int64_t)31;  // whole groups of 32 pairs
    chunk = std::min(chunk, n);
    if (chunk < 1)
        return SS_ERR_OOM;
    const size_t a_in = align_up((size_t)chunk * seq_in, 256);
    const size_t a_pk =
        format != SS_FMT_ASCII ? 0
        : sliced ? align_up((size_t)ss_sliced_words(m, chunk) * 4, 256)
                 : align_up((size_t)chunk * packed, 256);
    // per threshold, results at 16-byte aligned offsets
    const size_t acc_stride = align_up((size_t)chunk, 16);
    const size_t a_acc = align_up(acc_stride * n_e, 256);
    const size_t a_obs = align_up(acc_stride * 4 * n_e, 256);
    const size_t slot = 2 * a_in + 2 * a_pk + a_acc + a_obs;
    // the bucket area (thresholds beyond the plain kernel) sits first
    const size_t bws =
        all_plain ? 0 : align_up(ssk::bucket_ws_bytes(chunk), 256);
    if (bws + 2 * slot > ctx->budget)
        return SS_ERR_OOM;
    SS_TRY(ensure_workspace(ctx, bws + 2 * slot));
    for (int64_t p0 = 0, it = 0; p0 < n; p0 += chunk, ++it) {
        const int64_t cn = std::min(chunk, n - p0);
        const int sidx = (int)(it & 1);
        cudaStream_t st = ctx->hstream[sidx];
        char *base = (char *)ctx->ws + bws + sidx * slot;
        char *dq = base, *dr = base + a_in;
        uint32_t *pq = (uint32_t *)(base + 2 * a_in);
        uint32_t *pr = (uint32_t *)(base + 2 * a_in + a_pk);
        uint8_t *dacc = (uint8_t *)(base + 2 * a_in + 2 * a_pk);
        int32_t *dobs = (int32_t *)(base + 2 * a_in + 2 * a_pk + a_acc);
        const size_t in_bytes = (size_t)cn * seq_in;
        SS_CUDA(cudaMemcpyAsync(dq, (const char *)reads + p0 * seq_in,
                                in_bytes, cudaMemcpyHostToDevice, st));
        SS_CUDA(cudaMemcpyAsync(dr, (const char *)refs + p0 * seq_in,
                                in_bytes, cudaMemcpyHostToDevice, st));
        const uint32_t *fq = (const uint32_t *)dq, *fr = (const uint32_t *)dr;
        if (sliced) {
            SS_CUDA(ssk::launch_pack_sliced((const uint8_t *)dq, cn, m, pq,
                                            ctx->d_status, st));
            SS_CUDA(ssk::launch_pack_sliced((const uint8_t *)dr, cn, m, pr,
                                            ctx->d_status, st));
            ctx->counters.launches += 2;
        } else if (format == SS_FMT_ASCII) {
            SS_CUDA(ssk::launch_pack_fixed((const uint8_t *)dq, cn, m, pq,
                                           ctx->d_status, st));
            SS_CUDA(ssk::launch_pack_fixed((const uint8_t *)dr, cn, m, pr,
                                           ctx->d_status, st));
            ctx->counters.launches += 2;
            fq = pq;
            fr = pr;
        }
        if (sliced)
            SS_TRY(sweep_sliced(
                ctx, pq, pr, m, e_list, n_e, cn,
                [=](int t) { return dacc + (size_t)t * acc_stride; },
                [=](int t) { return dobs + (size_t)t * acc_stride; }, st));
        for (int t = 0; t < n_e; ++t) {
            uint8_t *ta = dacc + (size_t)t * acc_stride;
            int32_t *to = dobs + (size_t)t * acc_stride;
            if (sliced) {
                // filtered above
            } else if (m == 0) {
                SS_CUDA(cudaMemsetAsync(ta, 1, (size_t)cn, st));
                SS_CUDA(cudaMemsetAsync(to, 0, (size_t)cn * 4, st));
            } else {
                // the bucket area is shared: bucketed thresholds run on one
                // stream at a time, so wait for the other slot first
                if (!plain_ok(m, e_list[t]))
                    SS_CUDA(cudaStreamSynchronize(ctx->hstream[sidx ^ 1]));
                SS_TRY(filter_packed(ctx,
                                     make_pairs(fq, fr, nullptr, nullptr, m,
                                                nullptr, e_list[t], cn, ta,
                                                to),
                                     SS_FLAG_NO_GRAPH, st));
            }
            SS_CUDA(cudaMemcpyAsync(out_accept + (size_t)t * n + p0, ta,
                                    (size_t)cn, cudaMemcpyDeviceToHost, st));
            SS_CUDA(cudaMemcpyAsync(out_obstacles + (size_t)t * n + p0, to,
                                    (size_t)cn * 4, cudaMemcpyDeviceToHost,
                                    st));
        }
    }
    ctx->counters.pairs += n * n_e;
    SS_CUDA(cudaStreamSynchronize(ctx->hstream[0]));
    SS_CUDA(cudaStreamSynchronize(ctx->hstream[1]));
    return ss_sync(ctx, nullptr);
}

int ss_sync(ss_ctx *ctx, void *stream)
{
    if (!ctx)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(stream);
    SS_CUDA(cudaStreamSynchronize(st));
    SS_CUDA(cudaStreamSynchronize(ctx->stream));
    SS_CUDA(cudaStreamSynchronize(ctx->side));
    for (cudaStream_t l : ctx->lane)
        SS_CUDA(cudaStreamSynchronize(l));
    // take the status word (read and clear in one atomic exchange) on the
    // context's own non-blocking stream: a flag latched by a launch on any
    // other stream is either taken here or kept for the next ss_sync
    int flags = 0;
    SS_CUDA(ssk::launch_status_take(ctx->d_status, ctx->d_status + 1,
                                    ctx->stream));
    SS_CUDA(cudaMemcpyAsync(&flags, ctx->d_status + 1, sizeof(int),
                            cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(cudaStreamSynchronize(ctx->stream));
    if (flags) {
        if (flags & ssk::kStatusInvalidBase)
            return SS_ERR_INVALID_BASE;
        if (flags & ssk::kStatusInvalidArg)
            return SS_ERR_INVALID_ARG;
        if (flags & ssk::kStatusUnsupported)
            return SS_ERR_UNSUPPORTED;
        if (flags & ssk::kStatusTimeout)
            return SS_ERR_TIMEOUT;
    }
    return SS_OK;
}

int ss_check_wait_timeout(ss_ctx *ctx, int64_t limit_ns, void *stream)
{
    if (!ctx || limit_ns < 1000 || limit_ns > 10000000000LL)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(stream);
    SS_CUDA(ssk::launch_wait_timeout((uint64_t)limit_ns, ctx->d_status, st));
    ctx->counters.launches += 1;
    return SS_OK;
}

int ss_get_counters(const ss_ctx *ctx, ss_counters *out)
{
    if (!ctx || !out)
        return SS_ERR_INVALID_ARG;
    *out = ctx->counters;
    return SS_OK;
}

int ss_edit_distance_banded(ss_ctx *ctx, const void *reads, const void *refs,
                            int format, int32_t m, int32_t e, int64_t n,
                            void *stream, int32_t *out_ed)
{
    if (!ctx || n < 0 || m < 0 || e < 0)
        return SS_ERR_INVALID_ARG;
    if (format != SS_FMT_PACKED2)
        return SS_ERR_INVALID_ARG;
    if (e > ssk::kEdMaxE)
        return SS_ERR_UNSUPPORTED;
    if (n == 0)
        return SS_OK;
    if (!reads || !refs || !out_ed)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    SS_CUDA(ssk::launch_ed_banded(e, (const uint32_t *)reads,
                                  (const uint32_t *)refs, n, m, out_ed,
                                  ctx->sm_count, pick_stream(stream)));
    ctx->counters.launches += 1;
    return SS_OK;
}

int ss_filter_confusion(ss_ctx *ctx, const uint8_t *accept,
                        const int32_t *ed, int64_t n, int32_t e,
                        void *stream, uint64_t *out_counts)
{
    if (!ctx || n < 0 || e < 0 || !out_counts || (n > 0 && (!accept || !ed)))
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    SS_CUDA(ssk::launch_confusion(accept, ed, n, e,
                                  (unsigned long long *)out_counts,
                                  ctx->sm_count, pick_stream(stream)));
    ctx->counters.launches += 1;
    return SS_OK;
}

int ss_edit_distance_varlen(ss_ctx *ctx, const void *reads, const void *refs,
                            const int64_t *offsets, const int32_t *lengths,
                            const int32_t *E, int64_t n, void *stream,
                            int32_t *out_ed)
{
    if (!ctx || n < 0)
        return SS_ERR_INVALID_ARG;
    if (n == 0)
        return SS_OK;
    if (!reads || !refs || !offsets || !lengths || !E || !out_ed)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    SS_CUDA(ssk::launch_ed_var((const uint32_t *)reads,
                               (const uint32_t *)refs, offsets, lengths, E,
                               n, out_ed, ctx->d_status, ctx->sm_count,
                               pick_stream(stream)));
    ctx->counters.launches += 6;
    return SS_OK;
}

int ss_filter_unequal(ss_ctx *ctx, const void *reads, const int64_t *read_off,
                      const int32_t *read_len, const void *refs,
                      const int64_t *ref_off, const int32_t *ref_len,
                      const int32_t *E, int32_t e, int64_t n, void *stream,
                      uint8_t *out_accept, int32_t *out_obstacles)
{
    if (!ctx || n < 0 || (!E && e < 0))
        return SS_ERR_INVALID_ARG;
    if (n == 0)
        return SS_OK;
    if (!reads || !refs || !read_off || !read_len || !ref_off || !ref_len ||
        !out_accept || !out_obstacles)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(stream);
    SS_CUDA(ssk::launch_unequal((const uint32_t *)reads, read_off, read_len,
                                (const uint32_t *)refs, ref_off, ref_len, E,
                                e, n, out_accept, out_obstacles,
                                ctx->d_status, ctx->sm_count, st));
    ctx->counters.launches += 1;
    ctx->counters.pairs += n;
    return SS_OK;
}

int ss_filter_submaze(ss_ctx *ctx, const void *reads, const void *refs,
                      int format, int32_t m, int32_t e, int32_t t, int32_t y,
                      int64_t n, void *stream, uint8_t *out_accept,
                      int32_t *out_obstacles)
{
    if (!ctx || n < 0 || m < 0 || e < 0 || t < 1 || y < 1)
        return SS_ERR_INVALID_ARG;
    if (format != SS_FMT_PACKED2 && format != SS_FMT_SLICED2)
        return SS_ERR_INVALID_ARG;
    if (format == SS_FMT_SLICED2 ? e > ssk::kSlicedMaxE
                                 : ssk::eff_threshold(m, e) > 31)
        return SS_ERR_UNSUPPORTED;
    if (n == 0)
        return SS_OK;
    if (!reads || !refs || !out_accept || !out_obstacles)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(stream);
    if (m == 0) {
        SS_CUDA(cudaMemsetAsync(out_accept, 1, (size_t)n, st));
        SS_CUDA(cudaMemsetAsync(out_obstacles, 0, (size_t)n * 4, st));
        return SS_OK;
    }
    if (format == SS_FMT_SLICED2) {
        if ((((uintptr_t)reads) | ((uintptr_t)refs)) & 15)
            return SS_ERR_INVALID_ARG;
        SS_CUDA(ssk::launch_sliced_submaze((const uint32_t *)reads,
                                           (const uint32_t *)refs, n, m, e,
                                           t, y, out_accept, out_obstacles,
                                           st));
        ctx->counters.launches += 1;
        return SS_OK;
    }
    SS_CUDA(ssk::launch_submaze((const uint32_t *)reads,
                                (const uint32_t *)refs, n, m, e, t, y,
                                out_accept, out_obstacles, ctx->d_status,
                                ctx->sm_count, st));
    ctx->counters.launches += 1;
    return SS_OK;
}

int ss_compact_accepted(ss_ctx *ctx, const uint8_t *accept, int64_t n,
                        void *stream, int64_t *out_index, int64_t *out_count)
{
    if (!ctx || n < 0 || !out_count || (n > 0 && (!accept || !out_index)))
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    SS_TRY(ensure_workspace(ctx, ssk::compact_ws_bytes(n)));
    SS_CUDA(ssk::launch_compact(accept, n, (int64_t *)ctx->ws, out_index,
                                out_count, pick_stream(stream)));
    ctx->counters.launches += 3;
    return SS_OK;
}

int ss_gather_pairs(ss_ctx *ctx, const void *reads, const void *refs,
                    int32_t m, const int64_t *index, const int64_t *count,
                    int64_t n, void *stream, void *out_reads,
                    void *out_refs)
{
    if (!ctx || n < 0 || m < 0 || !count)
        return SS_ERR_INVALID_ARG;
    if (n > 0 && (!reads || !refs || !index || !out_reads || !out_refs))
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    SS_CUDA(ssk::launch_gather_pairs((const uint32_t *)reads,
                                     (const uint32_t *)refs, m, index, count,
                                     n, (uint32_t *)out_reads,
                                     (uint32_t *)out_refs, ctx->sm_count,
                                     pick_stream(stream)));
    ctx->counters.launches += 1;
    return SS_OK;
}

int ss_set_tuning(ss_ctx *ctx, int rw_max_e, int cw_subgrid)
{
    if (!ctx || (rw_max_e != 15 && rw_max_e != 31) ||
        (cw_subgrid != 4 && cw_subgrid != 8 && cw_subgrid != 16))
        return SS_ERR_INVALID_ARG;
    ctx->tune.rw_max_e = rw_max_e;
    ctx->tune.cw_subgrid = cw_subgrid;
    return SS_OK;
}

int ss_get_tuning(const ss_ctx *ctx, int *rw_max_e, int *cw_subgrid)
{
    if (!ctx || !rw_max_e || !cw_subgrid)
        return SS_ERR_INVALID_ARG;
    *rw_max_e = ctx->tune.rw_max_e;
    *cw_subgrid = ctx->tune.cw_subgrid;
    return SS_OK;
}

int ss_autotune(ss_ctx *ctx, const void *reads, const void *refs,
                const int64_t *offsets, const int32_t *lengths, int32_t m,
                const int32_t *E, int32_t e, int64_t n, void *stream,
                uint8_t *out_accept, int32_t *out_obstacles, int reps,
                float *best_ms)
{
    if (!ctx || n <= 0 || reps < 1 || !reads || !refs || !out_accept ||
        !out_obstacles || (offsets && !lengths) || (!lengths && m < 0) ||
        (!E && e < 0) || n > INT32_MAX)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(stream);
    SS_TRY(ensure_workspace(ctx, ssk::bucket_ws_bytes(n)));
    const ssk::PairSet ps = make_pairs(reads, refs, offsets, lengths, m, E, e,
                                       n, out_accept, out_obstacles);
    const ssk::TuneParams saved = ctx->tune;
    ssk::TuneParams best = saved;
    float best_t = 1e30f;
    cudaEvent_t a, z;
    SS_CUDA(cudaEventCreate(&a));
    SS_CUDA(cudaEventCreate(&z));
    int rc = SS_OK;
    for (int rmax : {15, 31}) {
        for (int k : {4, 8, 16}) {
            ctx->tune.rw_max_e = rmax;
            ctx->tune.cw_subgrid = k;
            rc = run_bucketed(ctx, ps, st, false);  // warm-up
            if (rc != SS_OK)
                break;
            cudaEventRecord(a, st);
            for (int r = 0; r < reps && rc == SS_OK; ++r)
                rc = run_bucketed(ctx, ps, st, false);
            cudaEventRecord(z, st);
            if (rc != SS_OK || cudaEventSynchronize(z) != cudaSuccess) {
                if (rc == SS_OK)
                    rc = SS_ERR_CUDA;
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, a, z);
            ms /= reps;
            if (ms < best_t) {
                best_t = ms;
                best = ctx->tune;
            }
        }
        if (rc != SS_OK)
            break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    ctx->tune = rc == SS_OK ? best : saved;
    if (best_ms)
        *best_ms = best_t;
    return rc;
}

}  // extern "C"
