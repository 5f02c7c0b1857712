// ss_internal.h -- host-side launch entry points of the kernels (not ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <utility>

#include "ss_rw_config.h"

namespace ssk {

struct RwUniformArgs;
struct RwLaunch;
struct PairSet;
struct BucketWs;
struct TuneParams;

cudaError_t launch_pack_fixed(const uint8_t *ascii, int64_t n, int32_t m,
                              uint32_t *out, int *status, cudaStream_t st);
cudaError_t launch_pack_varlen(const uint8_t *ascii, const int64_t *offsets,
                               const int32_t *lengths, int64_t n,
                               uint32_t *out, const int64_t *out_offsets,
                               int *status, int sm_count, cudaStream_t st,
                               uint8_t *bad_flags = nullptr);

// Bit-sliced layout (SS_FMT_SLICED2): fixed-stride ASCII -> sliced words
// (8 * ceil(m/4) * ceil(n/32) of them), and the plain launch over it for
// 0 <= E <= kSlicedMaxE.
constexpr int kSlicedMaxE = 31;
cudaError_t launch_pack_sliced(const uint8_t *ascii, int64_t n, int32_t m,
                               uint32_t *out, int *status, cudaStream_t st);
cudaError_t launch_sliced(const uint32_t *reads, const uint32_t *refs,
                          int64_t n, int32_t m, int32_t E, uint8_t *acc,
                          int32_t *obs, cudaStream_t st);
// The plain launch over up to kSlicedMaxSegments batches of one threshold E
// (each its own n >= 1 and m >= 0, sliced layout): one grid, the CTAs of
// segment s after those of segment s - 1.
struct SlicedSegment {
    const uint32_t *reads, *refs;
    int64_t n;
    int32_t m;       // read length (and reference length, equal lengths)
    uint8_t *acc;
    int32_t *obs;
    int32_t m_ref;   // reference length (launch_sliced_free_segments)
};
constexpr int kSlicedMaxSegments = 32;  // 2 KB of launch parameters
cudaError_t launch_sliced_segments(const SlicedSegment *segs, int nseg,
                                   int32_t E, cudaStream_t st);
// The same over batches whose reads and references differ in length
// (m != m_ref, both >= 0; reads in the sliced layout of m bases, refs of
// m_ref): Section 2.4's correction, a cell whose query base lies outside
// the read is free.
cudaError_t launch_sliced_free_segments(const SlicedSegment *segs, int nseg,
                                        int32_t E, cudaStream_t st);
// The sub-maze mode (sub-mazes of t columns, at most y segments each) over
// the bit-sliced layout, 0 <= E <= kSlicedMaxE.
cudaError_t launch_sliced_submaze(const uint32_t *reads, const uint32_t *refs,
                                  int64_t n, int32_t m, int32_t E, int32_t t,
                                  int32_t y, uint8_t *acc, int32_t *obs,
                                  cudaStream_t st);
// Several thresholds 0..4 in one pass (bit e of mask: threshold e; two or
// more bits): acc[i], obs[i] receive the i-th threshold of the mask in
// ascending order.
cudaError_t launch_sliced_set(const uint32_t *reads, const uint32_t *refs,
                              int64_t n, int32_t m, unsigned mask,
                              uint8_t *const *acc, int32_t *const *obs,
                              cudaStream_t st);

// K3a plain launch for 0 <= E <= kRwMaxE, m <= kRwMaxM.  status: device
// word for latched errors.
cudaError_t launch_rw_uniform(int E, const uint32_t *reads,
                              const uint32_t *refs, int64_t n, int32_t m,
                              uint8_t *acc, int32_t *obs, int *status,
                              cudaStream_t st);
// Devices the one-time set-up below keeps state for (ids 0..63).
constexpr int kMaxDevices = 64;
// Kernel attributes of the plain launches on device `device` (the current
// one; before any capture; called by bucket_init under its lock).
cudaError_t rw_init(int device);

// K2 + K4: bucketed persistent form of a mixed batch.
size_t bucket_ws_bytes(int64_t n);
BucketWs bucket_ws_at(void *base, int64_t n);
int cw_class_slice_words(int cls);
cudaError_t launch_bucketed_one_stream(const PairSet &ps, const BucketWs &ws,
                                       int *status, cudaStream_t st);
// Kernel attributes and persistent grid sizes of the current device, once
// per device (called by ss_create, ss_server_start and the allocation-free
// entry before any capture; safe to call from several host threads).
cudaError_t bucket_init();
// conditional: st is being captured; every class kernel goes into an IF
// node that the pass switches on only when its class has pairs.
// hook (serving only, never while capturing): the CTA-per-pair pairs that
// fit the long-pair queue's worker go into its ring (hook_expect of them)
// instead of the class kernels.  class_counts (kClasses entries, may be
// null): an upper bound of each class's pairs known on the host (pairs
// the queue takes not counted); classes bounded by 0 are not launched.
struct LongHook;
cudaError_t launch_bucketed(const PairSet &ps, const BucketWs &ws,
                            const TuneParams &tp, int *status, int sm_count,
                            cudaStream_t st, cudaStream_t side,
                            cudaEvent_t fork, cudaEvent_t join,
                            bool conditional, int *launches,
                            const LongHook *hook = nullptr,
                            int hook_expect = 0,
                            const int64_t *class_counts = nullptr);
// The first kernel of the pass (ss_seg.cu): uniform input tiles routed on
// the plain pipeline, the others classified and listed.
struct SegArgs;
size_t seg_smem_bytes();
cudaError_t launch_seg_direct(const SegArgs &a, cudaStream_t st);

// Accuracy harness (ss_verify.cu): banded edit distance, E <= kEdMaxE.
constexpr int kEdMaxE = 31;
cudaError_t launch_ed_banded(int E, const uint32_t *reads,
                             const uint32_t *refs, int64_t n, int32_t m,
                             int32_t *ed, int sm_count, cudaStream_t st);
// Warp per pair, any length, per-pair E <= kEdWarpMaxE.
constexpr int kEdWarpMaxE = 511;
cudaError_t launch_ed_var(const uint32_t *reads, const uint32_t *refs,
                          const int64_t *off, const int32_t *len,
                          const int32_t *E, int64_t n, int32_t *ed,
                          int *status, int sm_count, cudaStream_t st);
cudaError_t launch_confusion(const uint8_t *acc, const int32_t *ed,
                             int64_t n, int E, unsigned long long *counts,
                             int sm_count, cudaStream_t st);

// Sub-maze approximate mode (ss_submaze.cu), E' <= 31.
cudaError_t launch_submaze(const uint32_t *reads, const uint32_t *refs,
                           int64_t n, int32_t m, int32_t E, int32_t t,
                           int32_t y, uint8_t *acc, int32_t *obs,
                           int *status, int sm_count, cudaStream_t st);

// Pairs of different lengths (ss_unequal.cu).
cudaError_t launch_unequal(const uint32_t *reads, const int64_t *read_off,
                           const int32_t *read_len, const uint32_t *refs,
                           const int64_t *ref_off, const int32_t *ref_len,
                           const int32_t *E, int32_t e, int64_t n,
                           uint8_t *acc, int32_t *obs, int *status,
                           int sm_count, cudaStream_t st);

// Read and clear the status word in one atomic exchange; the old value
// lands in *taken (ss_selftest.cu).
cudaError_t launch_status_take(int *status, int *taken, cudaStream_t st);

// Bounded-wait self-test (ss_selftest.cu).
cudaError_t launch_wait_timeout(uint64_t limit_ns, int *status,
                                cudaStream_t st);

// Compaction of accepted pairs (ss_compact.cu).
size_t compact_ws_bytes(int64_t n);
cudaError_t launch_compact(const uint8_t *acc, int64_t n, int64_t *ws,
                           int64_t *out_index, int64_t *out_count,
                           cudaStream_t st);
cudaError_t launch_gather_pairs(const uint32_t *reads, const uint32_t *refs,
                                int32_t m, const int64_t *index,
                                const int64_t *count, int64_t n,
                                uint32_t *out_reads, uint32_t *out_refs,
                                int sm_count, cudaStream_t st);

// Per-translation-unit dispatchers (E ranges 0-9, 10-17, 18-24, 25-31).
cudaError_t launch_rw_uniform_e0(int E, const RwLaunch &L, cudaStream_t st);
cudaError_t launch_rw_uniform_e1(int E, const RwLaunch &L, cudaStream_t st);
cudaError_t launch_rw_uniform_e2(int E, const RwLaunch &L, cudaStream_t st);
cudaError_t launch_rw_uniform_e3(int E, const RwLaunch &L, cudaStream_t st);
cudaError_t rw_init_e0();
cudaError_t rw_init_e1();
cudaError_t rw_init_e2();
cudaError_t rw_init_e3();

}  // namespace ssk
