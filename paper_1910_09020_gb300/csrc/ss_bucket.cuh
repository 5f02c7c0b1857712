// ss_bucket.cuh -- K2: length/threshold buckets of a mixed batch, and the
// per-pair accessors shared by the bucketed kernels.
//
// Every pair is assigned to one class -- which kernel routes it -- from its
// length m and effective threshold E' = min(E, m-1) (rows with |s| >= m hold
// no Q base at all, so they are all obstacles and never bound the longest
// run; the count limit still uses E):
//   * RW  classes: E' <= 31, thread per pair, E' <= EMAX in {1, 3, 7, 15, 31}
//   * CWW classes: 32 <= E' <= 511 and m <= 16384, warp per pair, by m bound
//   * CWC classes: larger, CTA per pair, by CTA width and m bound
// Within a class pairs are ordered by length, longest first (quarter-octave
// bins), so that persistent workers take the biggest pairs first and a warp
// of the RW kernel sees similar lengths.
#pragma once
#include <cstdint>

#include "ss_rw_config.h"

namespace ssk {

constexpr int kRwClasses = 5;
__host__ __device__ constexpr int rw_emax(int c)
{
    return c == 0 ? 1 : c == 1 ? 3 : c == 2 ? 7 : c == 3 ? 15 : 31;
}
// m bounds of the warp-per-pair classes: a class's shared-memory slice is
// sized for its bound, so finer bounds put more CTAs on an SM (the kernel
// is latency-bound; its shared memory sets the CTAs per SM from 6 KB on)
constexpr int kCwwClasses = 7;
__host__ __device__ constexpr int cww_mbound(int c)
{
    return c == 0 ? 2048 : c == 1 ? 3072 : c == 2 ? 4096 : c == 3 ? 6144
         : c == 4 ? 8192 : c == 5 ? 12288 : 16384;
}
constexpr int kCwwMaxE = 511;
constexpr int kCwcWidths = 5;  // CTA widths 64, 128, 256, 512, 1024
constexpr int kCwcMbounds = 3;
__host__ __device__ constexpr int cwc_width(int w) { return 64 << w; }
__host__ __device__ constexpr int cwc_mbound(int b)
{
    return b == 0 ? 16384 : b == 1 ? 65536 : 131072;
}
constexpr int kMaxLen = 131072;  // longest pair the CW kernels stage
constexpr int kClasses = kRwClasses + kCwwClasses + kCwcWidths * kCwcMbounds;
constexpr int kLenBins = 72;
constexpr int kKeys = kClasses * kLenBins;

constexpr int kClassNone = -1;         // m == 0: answered directly
constexpr int kClassInvalid = -2;      // negative m or E
constexpr int kClassUnsupported = -3;  // too long for the staged kernels

__host__ __device__ inline int cwc_class(int w, int b)
{
    return kRwClasses + kCwwClasses + w * kCwcMbounds + b;
}

// Effective threshold: rows beyond |s| = m-1 cannot match.
__host__ __device__ inline int eff_threshold(int m, int E)
{
    return E < m - 1 ? E : (m > 0 ? m - 1 : 0);
}

__host__ __device__ inline int class_of(int m, int E)
{
    if (m < 0 || E < 0)
        return kClassInvalid;
    if (m == 0)
        return kClassNone;
    const int Ee = eff_threshold(m, E);
    if (Ee <= 31) {
        for (int c = 0; c < kRwClasses; ++c)
            if (Ee <= rw_emax(c))
                return c;
    }
    if (Ee <= kCwwMaxE && m <= cww_mbound(kCwwClasses - 1)) {
        for (int c = 0; c < kCwwClasses; ++c)
            if (m <= cww_mbound(c))
                return kRwClasses + c;
    }
    if (m > kMaxLen)
        return kClassUnsupported;
    const int words = (2 * Ee + 1 + 31) / 32;
    int w = 0;
    while (w < kCwcWidths - 1 && cwc_width(w) < words)
        ++w;
    int b = 0;
    while (m > cwc_mbound(b))
        ++b;
    return cwc_class(w, b);
}

// Knobs the autotuner picks (they change speed, never results):
//   rw_max_e   -- largest E' routed thread-per-pair (15 or 31); above it a
//                 pair goes to a warp (pairs per warp: 32 -> 1)
//   cw_subgrid -- columns evaluated bit-parallel across rows before the
//                 surviving runs are extended word-wise (4, 8 or 16)
struct TuneParams {
    int rw_max_e = 31;
    int cw_subgrid = 8;
};

__host__ __device__ inline int class_of_tuned(int m, int E,
                                              const TuneParams &tp)
{
    const int c = class_of(m, E);
    if (c >= 0 && c < kRwClasses && eff_threshold(m, E) > tp.rw_max_e) {
        // above the thread-per-pair limit: the warp or CTA kernel
        const int Ee = eff_threshold(m, E);
        (void)Ee;
        if (m <= cww_mbound(kCwwClasses - 1)) {
            for (int k = 0; k < kCwwClasses; ++k)
                if (m <= cww_mbound(k))
                    return kRwClasses + k;
        }
        int b = 0;
        while (m > cwc_mbound(b))
            ++b;
        return cwc_class(0, b);
    }
    return c;
}

// Quarter-octave length bin, counted from the longest (bin 0) down.
__host__ __device__ inline int len_bin_desc(int m)
{
    int lb = 0;
    for (int x = m; x > 1; x >>= 1)
        ++lb;  // ceil-ish log2 is fine: only the order matters
    int fine = lb >= 2 ? ((m >> (lb - 2)) & 3) : 0;
    int bin = 4 * lb + fine;
    if (bin > kLenBins - 1)
        bin = kLenBins - 1;
    return kLenBins - 1 - bin;
}

// The batch as the kernels see it.
struct PairSet {
    const uint32_t *reads;   // packed words
    const uint32_t *refs;
    const int64_t *offsets;  // word offset per pair, or NULL (fixed stride)
    const int32_t *lengths;  // per-pair m, or NULL (uniform m)
    const int32_t *Es;       // per-pair E, or NULL (uniform e)
    int32_t m, e;
    int64_t stride;          // words per pair when offsets == NULL
    int64_t n;
    uint8_t *acc;
    int32_t *obs;
    __device__ __forceinline__ int len(int64_t p) const
    {
        return lengths ? lengths[p] : m;
    }
    __device__ __forceinline__ int thr(int64_t p) const
    {
        return Es ? Es[p] : e;
    }
    __device__ __forceinline__ int64_t off(int64_t p) const
    {
        return offsets ? offsets[p] : p * stride;
    }
};

// Workspace of the bucketing pass (device).
struct BucketWs {
    int *hist;      // kKeys
    int *ndeferred; // tiles listed in deferred (zeroed with hist)
    int *cursor;    // kKeys
    int *ranges;    // 2 * kClasses: [begin, end) per class in perm
    unsigned *counters;  // kClasses work counters of the persistent kernels
    int32_t *deferred;   // input tiles (of kRwThreads pairs) left to the classes
    int32_t *perm;  // n pair indices, grouped by key
};

// The serving engine's device-resident queue of long pairs (ss_server.cu):
// a ring of entries that producers (the enqueue kernel of each batch's
// pass) fill and a long-lived worker kernel drains.  An entry is published
// by writing its seq (= ring position + 1) last; a consumer claims position
// h by moving head from h to h + 1 only once entry h carries seq h + 1.
struct LongEntry {
    int64_t pair;
    int32_t batch;
    uint32_t seq;
};

// One batch whose long pairs are queued: where its pairs and results live.
struct LongBatch {
    PairSet ps;
    const uint8_t *bad;  // per-pair invalid-input flags (routed as -1)
    int remaining;       // queued pairs not yet routed
    int gen;             // written to done[] when remaining reaches 0
};

struct LongQueue {
    LongEntry *ring;             // kLongRing entries
    unsigned long long *tail;    // positions reserved by producers
    unsigned long long *head;    // positions claimed by consumers
    unsigned long long *last;    // time of the last claim by any worker
    int *busy;                   // worker CTAs routing a pair now
    LongBatch *batches;          // kLongBatches descriptors
    volatile int *done;          // host-mapped: gen of each finished batch
    volatile int *stop;          // host-mapped: workers leave when set
};

constexpr int kLongRing = 1 << 18;   // entries (a power of two)
constexpr int kLongBatches = 64;     // descriptors
// Worker shape: one CTA of 512 threads per SM, split into two teams of
// 256 that each route their own pair, with 72 KB of shared memory each (the
// longest pair of the served workload, 100 kbp at E = 10^4, needs 70 KB).
// A/B on GB300, served workload at 2 slots (burst capacity): one pair per
// CTA of 256 threads 222k pairs/s, of 512 threads 260k; two teams with 48,
// 64, 72 and 80 KB each 342k, 25k, 374k and 376k -- with 48 KB the longest
// pairs stayed in their batches' passes, and with 64 KB those passes'
// kernels no longer fitted beside the worker and waited for it to leave;
// four teams of 128 threads with 24 KB each 222k.  768 or 1024 threads, or
// two CTAs per SM, left too little of the SM for the batches' own kernels.
constexpr int kLongThreads = 512;      // worker CTA width
constexpr int kLongCtasPerSm = 1;      // worker CTAs per SM
constexpr int kLongTeams = 2;          // pairs a worker CTA routes at once
constexpr int kLongWords = 36 * 1024;  // worker shared words per CTA

// Whether the queue takes a pair of class cls (m, E'): the CTA-per-pair
// classes whose staged planes fit the worker's shared memory.
__host__ __device__ inline bool long_queued(int cls, int m, int Ee);

// A batch's hook into the queue: its descriptor index, passed to the
// enqueue kernel of its pass.
struct LongHook {
    LongQueue q;
    int batch;
};

// Arguments of k_seg_direct (ss_seg.cu): groups of kSegGroup input tiles of
// kRwThreads pairs per CTA.
constexpr int kSegGroup = 8;
struct SegArgs {
    PairSet ps;
    BucketWs ws;
    TuneParams tp;
    int64_t ntiles;  // ceil(n / kRwThreads)
    uint32_t neg1;   // 0xffffffff (see rw_route)
    int *status;
};

}  // namespace ssk
