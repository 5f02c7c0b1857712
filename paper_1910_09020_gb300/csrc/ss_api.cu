// ss_api.cu -- the C ABI of include/ss.h: context, argument checks, workspace
// and kernel dispatch.  Every step of the filter runs in the CUDA kernels;
// this file only validates, allocates workspace and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "../../include/ss.h"
#include "ss_device.cuh"
#include "ss_internal.h"
#include "ss_rw.cuh"

struct ss_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t hstream[2] = {nullptr, nullptr};  // ss_filter_host pipeline
    int *d_status = nullptr;                        // latched device errors
    size_t budget = 0;
    // workspace: one growable device block
    void *ws = nullptr;
    size_t ws_bytes = 0;
    ss_counters counters{};
};

namespace {

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

// Grow the workspace to at least `bytes` (within the budget).  Only called
// outside of stream capture; the caller synchronises before a regrow.
int ensure_workspace(ss_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes)
        return SS_OK;
    if (bytes > ctx->budget)
        return SS_ERR_OOM;
    if (ctx->ws) {
        // the old block may still be read by work on any caller stream
        SS_CUDA(cudaDeviceSynchronize());
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
cudaStream_t pick_stream(ss_ctx *, void *stream)
{
    return (cudaStream_t)stream;
}

// Packed pairs, uniform m and E: the plain launch.
int filter_packed_uniform(ss_ctx *ctx, const uint32_t *reads,
                          const uint32_t *refs, int32_t m, int32_t e,
                          int64_t n, uint8_t *acc, int32_t *obs,
                          cudaStream_t st)
{
    if (e <= ssk::kRwMaxE && m <= ssk::kRwMaxM) {
        SS_CUDA(ssk::launch_rw_uniform(e, reads, refs, n, m, acc, obs, st));
        ctx->counters.launches += 1;
        return SS_OK;
    }
    return SS_ERR_UNSUPPORTED;
}

}  // namespace

namespace ssk {

cudaError_t launch_rw_uniform(int E, const uint32_t *reads,
                              const uint32_t *refs, int64_t n, int32_t m,
                              uint8_t *acc, int32_t *obs, cudaStream_t st)
{
    RwUniformArgs a;
    a.reads = reads;
    a.refs = refs;
    a.n = n;
    a.m = m;
    a.w16 = (m + 15) / 16;
    a.w16_magic = div_magic((uint32_t)std::max(a.w16, 1));
    a.acc = acc;
    a.obs = obs;
    const size_t smem =
        (size_t)2 * (size_t)std::max(a.w16, 1) * (kRwThreads + 1) * 4;
    const int64_t grid = (n + kRwThreads - 1) / kRwThreads;
    if (grid > 0x7fffffff)
        return cudaErrorInvalidValue;
    if (E <= 9)
        return launch_rw_uniform_e0(E, a, smem, (unsigned)grid, st);
    if (E <= 17)
        return launch_rw_uniform_e1(E, a, smem, (unsigned)grid, st);
    if (E <= 24)
        return launch_rw_uniform_e2(E, a, smem, (unsigned)grid, st);
    return launch_rw_uniform_e3(E, a, smem, (unsigned)grid, st);
}

}  // namespace ssk

extern "C" {

int ss_version(void) { return 100; }

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
        cudaStreamCreateWithFlags(&ctx->hstream[0], cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->hstream[1], cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        ss_destroy(ctx);
        return SS_ERR_CUDA;
    }
    ctx->sm_count = prop.multiProcessorCount;
    *out = ctx;
    return SS_OK;
}

int ss_destroy(ss_ctx *ctx)
{
    if (!ctx)
        return SS_OK;
    DeviceGuard g(ctx->device);
    if (ctx->stream)
        cudaStreamSynchronize(ctx->stream);
    for (cudaStream_t s : ctx->hstream)
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    if (ctx->ws)
        cudaFree(ctx->ws);
    if (ctx->d_status)
        cudaFree(ctx->d_status);
    if (ctx->stream)
        cudaStreamDestroy(ctx->stream);
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
    cudaStream_t st = pick_stream(ctx, stream);
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

int ss_filter_batch(ss_ctx *ctx, const void *reads, const void *refs,
                    int format, const int64_t *offsets,
                    const int32_t *lengths, int32_t m, const int32_t *E,
                    int32_t e, int64_t n, int flags, void *stream,
                    uint8_t *out_accept, int32_t *out_obstacles)
{
    (void)flags;
    if (!ctx || n < 0)
        return SS_ERR_INVALID_ARG;
    if (format != SS_FMT_ASCII && format != SS_FMT_PACKED2)
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
    cudaStream_t st = pick_stream(ctx, stream);
    ctx->counters.pairs += n;

    const bool uniform = !offsets && !lengths && !E;
    if (!uniform)
        return SS_ERR_UNSUPPORTED;  // bucketed path: added with K2/K4
    if (m == 0) {
        // nothing to route: every pair accepted with 0 obstacles
        SS_CUDA(cudaMemsetAsync(out_accept, 1, (size_t)n, st));
        SS_CUDA(cudaMemsetAsync(out_obstacles, 0, (size_t)n * 4, st));
        return SS_OK;
    }
    if (format == SS_FMT_PACKED2)
        return filter_packed_uniform(ctx, (const uint32_t *)reads,
                                     (const uint32_t *)refs, m, e, n,
                                     out_accept, out_obstacles, st);
    // ASCII: pack chunks into the workspace, then filter them.
    const int64_t w16 = (m + 15) / 16;
    const size_t per_pair = (size_t)2 * (size_t)w16 * 4;
    int64_t chunk = (int64_t)((ctx->budget - std::min<size_t>(ctx->budget, 1024)) / per_pair);
    if (chunk < 1)
        return SS_ERR_OOM;
    chunk = std::min(chunk, n);
    const size_t seq_bytes = align_up((size_t)chunk * w16 * 4, 256);
    int rc = ensure_workspace(ctx, 2 * seq_bytes);
    if (rc != SS_OK)
        return rc;
    uint32_t *pq = (uint32_t *)ctx->ws;
    uint32_t *pr = (uint32_t *)((char *)ctx->ws + seq_bytes);
    for (int64_t p0 = 0; p0 < n; p0 += chunk) {
        const int64_t cn = std::min(chunk, n - p0);
        const uint8_t *rq = (const uint8_t *)reads + p0 * (int64_t)m;
        const uint8_t *rr = (const uint8_t *)refs + p0 * (int64_t)m;
        SS_CUDA(ssk::launch_pack_fixed(rq, cn, m, pq, ctx->d_status, st));
        SS_CUDA(ssk::launch_pack_fixed(rr, cn, m, pr, ctx->d_status, st));
        ctx->counters.launches += 2;
        rc = filter_packed_uniform(ctx, pq, pr, m, e, cn, out_accept + p0,
                                   out_obstacles + p0, st);
        if (rc != SS_OK)
            return rc;
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
    for (int t = 0; t < n_e; ++t)
        if (e_list[t] < 0)
            return SS_ERR_INVALID_ARG;
    if (n == 0 || n_e == 0)
        return SS_OK;
    if (!reads || !refs || !out_accept || !out_obstacles)
        return SS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok)
        return SS_ERR_CUDA;
    const int64_t w16 = (m + 15) / 16;
    // bytes of one sequence in the input format
    const size_t seq_in = format == SS_FMT_ASCII ? (size_t)m : (size_t)w16 * 4;
    const size_t packed = (size_t)w16 * 4;
    const size_t per_pair = 2 * seq_in +
                            (format == SS_FMT_ASCII ? 2 * packed : 0) +
                            (size_t)n_e * 5;
    // two pipeline slots, each holding one chunk
    int64_t chunk = (int64_t)(ctx->budget / (2 * per_pair + 1024));
    chunk = std::min<int64_t>(chunk, (int64_t)1 << 22);
    chunk = std::min(chunk, n);
    if (chunk < 1)
        return SS_ERR_OOM;
    const size_t a_in = align_up((size_t)chunk * seq_in, 256);
    const size_t a_pk =
        format == SS_FMT_ASCII ? align_up((size_t)chunk * packed, 256) : 0;
    const size_t a_acc = align_up((size_t)chunk * n_e, 256);
    const size_t a_obs = align_up((size_t)chunk * 4 * n_e, 256);
    const size_t slot = 2 * a_in + 2 * a_pk + a_acc + a_obs;
    int rc = ensure_workspace(ctx, 2 * slot);
    if (rc != SS_OK)
        return rc;
    for (int64_t p0 = 0, it = 0; p0 < n; p0 += chunk, ++it) {
        const int64_t cn = std::min(chunk, n - p0);
        const int sidx = (int)(it & 1);
        cudaStream_t st = ctx->hstream[sidx];
        char *base = (char *)ctx->ws + sidx * slot;
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
        if (format == SS_FMT_ASCII) {
            SS_CUDA(ssk::launch_pack_fixed((const uint8_t *)dq, cn, m, pq,
                                           ctx->d_status, st));
            SS_CUDA(ssk::launch_pack_fixed((const uint8_t *)dr, cn, m, pr,
                                           ctx->d_status, st));
            ctx->counters.launches += 2;
            fq = pq;
            fr = pr;
        }
        for (int t = 0; t < n_e; ++t) {
            uint8_t *ta = dacc + (size_t)t * cn;
            int32_t *to = dobs + (size_t)t * cn;
            if (m == 0) {
                SS_CUDA(cudaMemsetAsync(ta, 1, (size_t)cn, st));
                SS_CUDA(cudaMemsetAsync(to, 0, (size_t)cn * 4, st));
            } else {
                rc = filter_packed_uniform(ctx, fq, fr, m, e_list[t], cn, ta,
                                           to, st);
                if (rc != SS_OK)
                    return rc;
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
    cudaStream_t st = pick_stream(ctx, stream);
    SS_CUDA(cudaStreamSynchronize(st));
    SS_CUDA(cudaStreamSynchronize(ctx->stream));
    int flags = 0;
    SS_CUDA(cudaMemcpy(&flags, ctx->d_status, sizeof(int),
                       cudaMemcpyDeviceToHost));
    if (flags) {
        SS_CUDA(cudaMemset(ctx->d_status, 0, sizeof(int)));
        if (flags & ssk::kStatusInvalidBase)
            return SS_ERR_INVALID_BASE;
        if (flags & ssk::kStatusInvalidArg)
            return SS_ERR_INVALID_ARG;
        if (flags & ssk::kStatusTimeout)
            return SS_ERR_TIMEOUT;
    }
    return SS_OK;
}

int ss_get_counters(const ss_ctx *ctx, ss_counters *out)
{
    if (!ctx || !out)
        return SS_ERR_INVALID_ARG;
    *out = ctx->counters;
    return SS_OK;
}

}  // extern "C"
