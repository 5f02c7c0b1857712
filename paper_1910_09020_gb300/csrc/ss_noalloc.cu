// ss_noalloc.cu -- the allocation-free variant of the bucketed filter.
//
// Some callers cannot allocate device memory: a service that reserves all
// of a GPU's memory up front through its own allocator (an extra cudaMalloc
// would fail, or would synchronise the device at an unpredictable moment),
// or a plug-in running inside another program that must stay within that
// program's memory.  ss_filter_batch_noalloc() gives them the bucketed
// filter without a context and without any allocation: its scratch (the
// class histogram, scan cursors, class ranges, work counters and the pair
// permutation) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads this library holds until the process exits.
//
// The array's name in host code is only a stand-in for the device symbol,
// so the first call on each device -- with that device current -- looks up
// its device address with cudaGetSymbolAddress (and sizes the persistent
// grids); later calls reuse it.  Every call shares the one array: calls
// that overlap on the GPU (other streams, other host threads) race on it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/ss.h"
#include "ss_bucket.cuh"
#include "ss_internal.h"

namespace {

// Bucket workspace for SS_NOALLOC_MAX_PAIRS pairs (4 B of permutation per
// pair plus the class tables) and, at the end, the word the kernels latch
// their status flags into.  This entry point reports no status (bad pairs
// are marked by obstacles = -1 instead), so that word is a sink nothing
// reads and needs no clearing.
constexpr size_t kScratchBytes = (size_t)4 * SS_NOALLOC_MAX_PAIRS + 64 * 1024;
constexpr size_t kStatusOffset = kScratchBytes - 256;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

using ssk::kMaxDevices;
struct DeviceSetup {
    bool ready = false;
    void *scratch = nullptr;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Device address of the scratch array on the current device (set up once).
int scratch_of_current_device(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return SS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices)
        return SS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (!s.ready) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess ||
            ptr == nullptr) {
            (void)cudaGetLastError();
            return SS_ERR_CUDA;
        }
        if (ssk::bucket_init() != cudaSuccess) {
            (void)cudaGetLastError();
            return SS_ERR_CUDA;
        }
        s.scratch = ptr;
        s.ready = true;
    }
    *out = s.scratch;
    return SS_OK;
}

}  // namespace

extern "C" int ss_filter_batch_noalloc(const void *reads, const void *refs,
                                       const int64_t *offsets,
                                       const int32_t *lengths, int32_t m,
                                       const int32_t *E, int32_t e, int64_t n,
                                       void *stream, uint8_t *out_accept,
                                       int32_t *out_obstacles)
{
    if (n < 0)
        return SS_ERR_INVALID_ARG;
    if (n == 0)
        return SS_OK;
    if (!reads || !refs || !out_accept || !out_obstacles)
        return SS_ERR_INVALID_ARG;
    if (offsets && !lengths)
        return SS_ERR_INVALID_ARG;
    if ((!lengths && m < 0) || (!E && e < 0))
        return SS_ERR_INVALID_ARG;
    if (n > SS_NOALLOC_MAX_PAIRS)
        return SS_ERR_OOM;  // beyond the fixed scratch
    if (ssk::bucket_ws_bytes(n) + 256 > kStatusOffset)
        return SS_ERR_OOM;
    void *scratch = nullptr;
    const int rc = scratch_of_current_device(&scratch);
    if (rc != SS_OK)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int *status = (int *)((char *)scratch + kStatusOffset);
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
    ps.acc = out_accept;
    ps.obs = out_obstacles;
    const ssk::BucketWs ws = ssk::bucket_ws_at(scratch, n);
    if (ssk::launch_bucketed_one_stream(ps, ws, status, st) != cudaSuccess) {
        (void)cudaGetLastError();
        return SS_ERR_CUDA;
    }
    return SS_OK;
}
