// ss_server.cu -- continuous-batching request server over the bucketed
// filter (not in the paper, whose GPU version filters one prepared batch).
//
// Clients submit requests (host ASCII pairs with per-pair lengths and
// thresholds).  A scheduler thread keeps up to `slots` batches in flight:
// whenever a slot is free it admits pending requests first-in first-out
// while their device footprint fits the HBM budget, copies them to the
// device (batch memory comes from a memory pool of the server's own), packs
// them, and runs the bucketed pass with persistent grids sized to 1/slots
// of the SMs, so that a batch admitted while others run executes beside
// them instead of queueing behind them.
//
// Long pairs do not hold a slot.  The pairs of the CTA-per-pair classes
// (thresholds above 511, or reads past 16 kbp) that fit the worker's shared
// memory go into a device-resident ring instead of their batch's class
// kernels, and one long-lived persistent worker kernel (one CTA per SM)
// drains that ring for every batch: a slot frees as soon as its pass ends,
// while its long pairs run beside later batches' work.  The worker exits
// after a bounded idle time (or when the server stops) and the scheduler
// relaunches it while queued pairs remain; its waits on the ring are
// bounded.  A batch is done when its pass has ended (a host-function
// callback on its stream) and its last queued pair is routed (the worker
// that routes it writes the batch's generation into host-mapped memory).
// Results stay in device memory until the client fetches them.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ss.h"
#include "ss_bucket.cuh"
#include "ss_cw.cuh"
#include "ss_device.cuh"
#include "ss_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(Clock::now().time_since_epoch())
        .count();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

enum ReqState { kPending = 0, kRunning = 1, kDone = 2 };

struct Batch;

struct Request {
    uint64_t id = 0;
    const uint8_t *reads = nullptr, *refs = nullptr;  // caller-owned, host
    std::vector<int32_t> lengths, E;
    std::vector<int64_t> offsets;  // byte offset of each pair in reads/refs
    int64_t n = 0;
    int64_t bases = 0;
    size_t footprint = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    int state = kPending;
    int status = SS_OK;
    std::shared_ptr<Batch> batch;  // holds the device results
    int64_t first = 0;             // first pair of this request in the batch
};

struct Batch {
    int slot = -1;
    std::vector<Request *> reqs;
    int64_t n = 0;
    void *dev = nullptr;   // inputs + workspace + results of the batch
    size_t bytes = 0;
    uint8_t *acc = nullptr;
    int32_t *obs = nullptr;
    int *status = nullptr;
    uint8_t *bad = nullptr;         // per-pair invalid-input flags (device)
    std::vector<uint8_t> host_bad;  // copied back at completion
    cudaStream_t st = nullptr;
    int pinned_refs = 0;   // requests whose results are still unfetched
    std::atomic<bool> done{false};
    double t_done = 0;
    std::vector<char> host_meta;  // staging of offsets/lengths/E
    // long-pair queue: descriptor index (-1: none queued), generation,
    // queued pairs, and the descriptor's host staging
    int lq_batch = -1;
    int lq_gen = 0;
    int64_t nlong = 0;
    ssk::LongBatch lq_desc{};
    bool pass_seen = false;  // the pass ended (slot released)
};

struct Slot {
    cudaStream_t st = nullptr, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    std::shared_ptr<Batch> running;
};

}  // namespace

struct ss_server {
    int device = 0;
    int sm_count = 0;
    int nslots = 2;
    size_t budget = 0;
    size_t in_use = 0;
    std::vector<Slot> slots;
    // reads of results and status words: a non-blocking stream, so a read
    // waits for nothing the caller has queued on the legacy default stream
    cudaStream_t copy_st = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread thread;
    int64_t max_batch_pairs = 1 << 20;
    cudaMemPool_t pool = nullptr;  // the server's own batch memory
    // long-pair queue: device ring, counters and descriptors (lq_dev),
    // host-mapped done flags and stop word (lq_host), the worker's stream
    ssk::LongQueue lq{};
    void *lq_dev = nullptr;
    int *lq_host = nullptr;
    cudaStream_t wst = nullptr;
    cudaEvent_t wev = nullptr;
    bool worker_launched = false;
    std::vector<int> lq_free;        // free descriptor indices
    int lq_gen = 0;
    int64_t lq_inflight = 0;         // queued pairs not yet routed
    std::vector<std::shared_ptr<Batch>> draining;  // pass ended, long pairs left
    // statistics
    std::vector<double> latencies;
    int64_t done_requests = 0, done_pairs = 0, done_bases = 0;
    int64_t batches = 0, max_inflight_seen = 0;
    int64_t long_queued = 0, worker_launches = 0;
    double t_first_submit = 0, t_last_done = 0;
    int sticky_error = SS_OK;
};

namespace {

// Device -> host read on the server's copy stream (the batch it reads from
// has completed).
cudaError_t read_back(ss_server *s, void *dst, const void *src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost,
                                    s->copy_st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s->copy_st);
    return e;
}

// Device bytes a request needs while it runs (inputs, packed words,
// per-pair metadata, bucket permutation, results).
size_t footprint_of(const Request &r)
{
    size_t words = 0;
    for (int32_t m : r.lengths)
        words += (size_t)(m + 15) / 16;
    return 2 * (size_t)r.bases + 2 * 4 * words + (size_t)r.n * (8 + 8 + 4 + 4 + 4 + 1 + 4) + 4096;
}

// Pairs whose input held a non-base are answered (accept 0, obstacles -1)
// after routing, so a bad request fails alone.
__global__ void k_mark_bad(const uint8_t *__restrict__ bad, int64_t n,
                           uint8_t *acc, int32_t *obs)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        if (bad[p]) {
            acc[p] = 0;
            obs[p] = -1;
        }
}

// The worker's idle bound: it leaves after this long without a queued pair
// (long enough to stay through the gaps between requests under load).
constexpr uint64_t kWorkerIdleNs = 100000000ull;  // 100 ms
constexpr uint32_t kWorkerMaxPolls = 1u << 22;

// Claim the next published entry of the ring: its batch (>= 0) and pair,
// or -1 once no worker CTA is routing a pair and none has claimed one for
// idle_ns (or after kWorkerMaxPolls polls), or the server asked the workers
// to stop.  So the CTAs leave together: one that left while others still
// route long pairs would shrink a kernel that keeps running, and the host
// relaunches only a finished one.  A successful claim counts the CTA busy
// (the caller ends that with long_done).
__device__ int long_claim(const ssk::LongQueue &q, uint64_t idle_ns,
                          int64_t &pair)
{
    uint64_t t0 = 0;
    uint32_t sleep_ns = 32;
    for (uint32_t polls = 0; polls < kWorkerMaxPolls; ++polls) {
        if (*q.stop)
            return -1;
        const unsigned long long h =
            *(volatile unsigned long long *)q.head;
        const ssk::LongEntry *e = q.ring + (h & (ssk::kLongRing - 1));
        const uint32_t seq = *(volatile const uint32_t *)&e->seq;
        if (seq == (uint32_t)(h + 1)) {
            if (atomicCAS(q.head, h, h + 1) == h) {
                *(volatile unsigned long long *)q.last = ssk::global_ns();
                atomicAdd(q.busy, 1);
                __threadfence();
                pair = *(volatile const int64_t *)&e->pair;
                return *(volatile const int32_t *)&e->batch;
            }
            continue;  // another CTA took it: try the next one at once
        }
        const uint64_t now = ssk::global_ns();
        if (t0 == 0)
            t0 = now;
        const uint64_t last = *(volatile unsigned long long *)q.last;
        const uint64_t since = last > t0 ? last : t0;
        if (now > since && now - since > idle_ns &&
            *(volatile int *)q.busy == 0)
            return -1;
        __nanosleep(sleep_ns);
        if (sleep_ns < 4096)
            sleep_ns *= 2;
    }
    return -1;
}

// The long-lived worker: each CTA is two teams of 256 threads, and each
// team takes queued pairs one at a time and routes each (Section 2.4, rows
// across the team's threads) in its half of the shared memory;
// the team that routes a batch's last queued pair publishes the batch's
// generation to the host.  Pairs flagged as holding a non-base get
// obstacles -1 (their batch's request fails alone, as in the pass).
__global__ void __launch_bounds__(ssk::kLongThreads)
    k_long_worker(const ssk::LongQueue q, uint64_t idle_ns)
{
    constexpr int TT = ssk::kLongThreads / ssk::kLongTeams;
    extern __shared__ uint32_t smem[];
    __shared__ int red[ssk::kLongTeams][2][32];
    __shared__ int64_t s_pair[ssk::kLongTeams];
    __shared__ int s_batch[ssk::kLongTeams];
    const int team = threadIdx.x / TT, t = threadIdx.x % TT;
    const int bar = 1 + team;  // named barrier of the team
    uint32_t *slice = smem + team * (ssk::kLongWords / ssk::kLongTeams);
    int buf = 0;
    for (;;) {
        if (t == 0) {
            int64_t p = 0;
            s_batch[team] = long_claim(q, idle_ns, p);
            s_pair[team] = p;
        }
        ssk::team_sync(bar, TT);
        const int b = s_batch[team];
        if (b < 0)
            break;
        const int64_t p = s_pair[team];
        const ssk::PairSet ps = q.batches[b].ps;
        const uint8_t *bad = q.batches[b].bad;
        const int m = ps.len(p), E = ps.thr(p);
        int count = -1;
        if (!(bad && bad[p])) {
            const int64_t off = ps.off(p);
            count = ssk::cw_team_route<8>(slice, red[team], buf,
                                          ps.reads + off, ps.refs + off, m, E,
                                          t, TT, bar);
        }
        if (t == 0) {
            ps.acc[p] = (uint8_t)(count >= 0 && count <= E);
            ps.obs[p] = count;
            __threadfence();
            if (atomicSub(&q.batches[b].remaining, 1) == 1) {
                __threadfence_system();
                q.done[b] = q.batches[b].gen;
                __threadfence_system();
            }
            atomicSub(q.busy, 1);
        }
        ssk::team_sync(bar, TT);  // the slice and s_batch are reused
    }
}

size_t worker_smem() { return (size_t)ssk::kLongWords * 4; }

// Launch the worker if work is in flight (want, or queued pairs remain)
// and none is running.  It is launched ahead of each batch's kernels: its
// CTAs need a share of every SM that the batches' persistent grids would
// otherwise fill.
void ensure_worker(ss_server *s, bool want = false)
{
    if (!want && s->lq_inflight <= 0)
        return;
    if (s->worker_launched && cudaEventQuery(s->wev) == cudaErrorNotReady)
        return;
    (void)cudaGetLastError();
    k_long_worker<<<s->sm_count * ssk::kLongCtasPerSm, ssk::kLongThreads,
                    worker_smem(), s->wst>>>(s->lq, kWorkerIdleNs);
    if (cudaGetLastError() != cudaSuccess ||
        cudaEventRecord(s->wev, s->wst) != cudaSuccess) {
        (void)cudaGetLastError();
        s->sticky_error = SS_ERR_CUDA;
        return;
    }
    s->worker_launched = true;
    s->worker_launches += 1;
}

void CUDART_CB on_batch_done(void *arg)
{
    Batch *b = (Batch *)arg;
    b->t_done = now_s();
    b->done.store(true, std::memory_order_release);
}

// Launch one batch on a free slot.  Called with the server lock held.
int launch_batch(ss_server *s, int slot_idx, std::vector<Request *> &take)
{
    Slot &sl = s->slots[slot_idx];
    auto b = std::make_shared<Batch>();
    b->slot = slot_idx;
    b->reqs = take;
    int64_t n = 0, bases = 0;
    size_t words = 0;
    for (Request *r : take) {
        r->first = n;
        n += r->n;
        bases += r->bases;
        for (int32_t m : r->lengths)
            words += (size_t)(m + 15) / 16;
    }
    b->n = n;
    // device layout: [bucket ws][ascii Q][ascii R][packed Q][packed R]
    //                [byte off][word off][lengths][E][acc][obs][status]
    const size_t a_ws = align_up(ssk::bucket_ws_bytes(n), 256);
    const size_t a_ascii = align_up((size_t)std::max<int64_t>(bases, 1), 256);
    const size_t a_pk = align_up(std::max<size_t>(words, 1) * 4, 256);
    const size_t a_i64 = align_up((size_t)n * 8, 256);
    const size_t a_i32 = align_up((size_t)n * 4, 256);
    const size_t a_u8 = align_up((size_t)n, 256);
    b->bytes = a_ws + 2 * a_ascii + 2 * a_pk + 2 * a_i64 + 2 * a_i32 +
               2 * a_u8 + a_i32 + 256;
    if (cudaMallocFromPoolAsync(&b->dev, b->bytes, s->pool, sl.st) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return SS_ERR_OOM;
    }
    char *p = (char *)b->dev;
    void *ws = p;
    p += a_ws;
    uint8_t *dq = (uint8_t *)p;
    p += a_ascii;
    uint8_t *dr = (uint8_t *)p;
    p += a_ascii;
    uint32_t *pq = (uint32_t *)p;
    p += a_pk;
    uint32_t *pr = (uint32_t *)p;
    p += a_pk;
    int64_t *boff = (int64_t *)p;
    p += a_i64;
    int64_t *woff = (int64_t *)p;
    p += a_i64;
    int32_t *dlen = (int32_t *)p;
    p += a_i32;
    int32_t *dE = (int32_t *)p;
    p += a_i32;
    b->acc = (uint8_t *)p;
    p += a_u8;
    b->obs = (int32_t *)p;
    p += a_i32;
    b->bad = (uint8_t *)p;
    p += a_u8;
    b->status = (int *)p;
    b->st = sl.st;

    // host metadata of the batch (staged once, copied in one transfer each)
    b->host_meta.resize((size_t)n * (8 + 8 + 4 + 4));
    int64_t *h_boff = (int64_t *)b->host_meta.data();
    int64_t *h_woff = h_boff + n;
    int32_t *h_len = (int32_t *)(h_woff + n);
    int32_t *h_E = h_len + n;
    int64_t bo = 0, wo = 0, i = 0;
    for (Request *r : take) {
        for (int64_t k = 0; k < r->n; ++k, ++i) {
            h_boff[i] = bo + r->offsets[k];
            h_woff[i] = wo;
            h_len[i] = r->lengths[k];
            h_E[i] = r->E[k];
            wo += (r->lengths[k] + 15) / 16;
        }
        bo += r->bases;
    }
    cudaStream_t st = sl.st;
    cudaError_t e = cudaSuccess;
    // inputs: one copy per request and sequence set
    int64_t at = 0;
    for (Request *r : take) {
        if (r->bases > 0) {
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dq + at, r->reads, (size_t)r->bases,
                                    cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dr + at, r->refs, (size_t)r->bases,
                                    cudaMemcpyHostToDevice, st);
        }
        at += r->bases;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(boff, h_boff, (size_t)n * 8,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(woff, h_woff, (size_t)n * 8,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dlen, h_len, (size_t)n * 4,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dE, h_E, (size_t)n * 4, cudaMemcpyHostToDevice,
                            st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->status, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->bad, 0, (size_t)n, st);
    if (e == cudaSuccess)
        e = ssk::launch_pack_varlen(dq, boff, dlen, n, pq, woff, b->status,
                                    s->sm_count, st, b->bad);
    if (e == cudaSuccess)
        e = ssk::launch_pack_varlen(dr, boff, dlen, n, pr, woff, b->status,
                                    s->sm_count, st, b->bad);
    ssk::PairSet ps;
    ps.reads = pq;
    ps.refs = pr;
    ps.offsets = woff;
    ps.lengths = dlen;
    ps.Es = dE;
    ps.m = 0;
    ps.e = 0;
    ps.stride = 0;
    ps.n = n;
    ps.acc = b->acc;
    ps.obs = b->obs;
    int launches = 0;
    const int share = std::max(1, s->sm_count / s->nslots);
    ensure_worker(s, true);
    // the long pairs the queue takes (the device's enqueue applies the
    // same rule), if a descriptor and ring room are free
    // and the pairs of every class (the pass launches only the classes
    // that have some: an empty class kernel of the CTA-per-pair classes
    // would still wait for shared memory beside the queue's worker)
    int64_t nlong = 0;
    std::vector<int64_t> counts(ssk::kClasses, 0), queued(ssk::kClasses, 0);
    {
        const ssk::TuneParams tp;
        for (int64_t k = 0; k < n; ++k) {
            const int m = h_len[k], E = h_E[k];
            const int cls = ssk::class_of_tuned(m, E, tp);
            if (cls < 0)
                continue;
            counts[cls] += 1;
            if (ssk::long_queued(cls, m, ssk::eff_threshold(m, E))) {
                queued[cls] += 1;
                ++nlong;
            }
        }
    }
    ssk::LongHook hook;
    const ssk::LongHook *hp = nullptr;
    if (nlong > 0 && !s->lq_free.empty() &&
        s->lq_inflight + nlong <= ssk::kLongRing) {
        for (int c = 0; c < ssk::kClasses; ++c)
            counts[c] -= queued[c];
        b->lq_batch = s->lq_free.back();
        s->lq_free.pop_back();
        b->lq_gen = ++s->lq_gen;
        b->nlong = nlong;
        b->lq_desc.ps = ps;
        b->lq_desc.bad = b->bad;
        b->lq_desc.remaining = (int)nlong;
        b->lq_desc.gen = b->lq_gen;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->lq.batches + b->lq_batch, &b->lq_desc,
                                sizeof(ssk::LongBatch),
                                cudaMemcpyHostToDevice, st);
        hook.q = s->lq;
        hook.batch = b->lq_batch;
        hp = &hook;
    }
    if (e == cudaSuccess)
        e = ssk::launch_bucketed(ps, ssk::bucket_ws_at(ws, n), ssk::TuneParams(),
                                 b->status, share, st, sl.side, sl.fork,
                                 sl.join, false, &launches, hp,
                                 hp ? (int)nlong : 0, counts.data());
    if (e == cudaSuccess) {
        const int g = (int)std::min<int64_t>((n + 255) / 256, 4 * s->sm_count);
        k_mark_bad<<<g, 256, 0, st>>>(b->bad, n, b->acc, b->obs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaLaunchHostFunc(st, on_batch_done, b.get());
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        cudaStreamSynchronize(st);
        cudaFreeAsync(b->dev, st);
        // a descriptor whose enqueue may have run is not reused
        return SS_ERR_CUDA;
    }
    if (b->nlong > 0) {
        s->lq_inflight += b->nlong;
        s->long_queued += b->nlong;
    }
    const double t = now_s();
    for (Request *r : take) {
        r->state = kRunning;
        r->t_start = t;
        r->batch = b;
    }
    b->pinned_refs = (int)take.size();
    sl.running = b;
    s->batches += 1;
    return SS_OK;
}

// Release the device memory of a batch whose results are all fetched.
void maybe_free_batch(ss_server *s, const std::shared_ptr<Batch> &b)
{
    if (b->pinned_refs == 0 && b->dev) {
        cudaFreeAsync(b->dev, b->st);  // back to the stream-ordered pool
        b->dev = nullptr;
        s->in_use -= std::min(s->in_use, b->bytes);
    }
}

// A batch whose pass has ended and whose queued pairs are all routed:
// read its status words and complete its requests.  Lock held.
void finish_batch(ss_server *s, const std::shared_ptr<Batch> &b, double t_done)
{
    int dev_status = 0;
    int st = SS_OK;
    if (read_back(s, &dev_status, b->status, sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        st = SS_ERR_CUDA;
    }
    // a bad base fails its own request only
    if (dev_status & ssk::kStatusInvalidBase) {
        b->host_bad.resize((size_t)b->n);
        if (read_back(s, b->host_bad.data(), b->bad, (size_t)b->n) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            st = SS_ERR_CUDA;
        }
    }
    if (st == SS_OK && (dev_status & ssk::kStatusUnsupported))
        st = SS_ERR_UNSUPPORTED;
    for (Request *r : b->reqs) {
        r->state = kDone;
        r->status = st;
        if (!b->host_bad.empty())
            for (int64_t k = 0; k < r->n; ++k)
                if (b->host_bad[(size_t)(r->first + k)]) {
                    r->status = SS_ERR_INVALID_BASE;
                    break;
                }
        r->t_done = t_done;
        s->latencies.push_back(r->t_done - r->t_submit);
        s->done_requests += 1;
        s->done_pairs += r->n;
        s->done_bases += r->bases;
    }
    s->t_last_done = std::max(s->t_last_done, t_done);
    if (b->lq_batch >= 0) {
        s->lq_free.push_back(b->lq_batch);
        s->lq_inflight -= b->nlong;
        b->lq_batch = -1;
    }
}

// The queued pairs of batch b are all routed (the worker published its
// generation to the host-mapped done word).
bool drained(const ss_server *s, const Batch &b)
{
    return b.lq_batch < 0 ||
           ((volatile const int *)s->lq_host)[b.lq_batch] == b.lq_gen;
}

void scheduler(ss_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (!s->stop) {
        // completions: a slot frees when its pass ends; the batch completes
        // once its queued long pairs are routed as well
        bool any_done = false;
        for (Slot &sl : s->slots) {
            std::shared_ptr<Batch> b = sl.running;
            if (!b || !b->done.load(std::memory_order_acquire))
                continue;
            sl.running.reset();
            b->pass_seen = true;
            s->draining.push_back(b);
        }
        for (size_t i = 0; i < s->draining.size();) {
            std::shared_ptr<Batch> b = s->draining[i];
            if (!drained(s, *b)) {
                ++i;
                continue;
            }
            finish_batch(s, b, std::max(b->t_done, b->nlong ? now_s() : 0.0));
            s->draining.erase(s->draining.begin() + (long)i);
            any_done = true;
        }
        if (any_done)
            s->cv_done.notify_all();
        bool busy = !s->pending.empty() || !s->draining.empty();
        for (const Slot &sl : s->slots)
            busy |= (bool)sl.running;
        ensure_worker(s, busy);
        // admission: fill free slots first-in first-out within the budget;
        // a backlog is shared out over all free slots (by pairs), so a
        // burst runs on every slot instead of queueing as one batch
        int free_slots = 0;
        for (const Slot &sl : s->slots)
            free_slots += sl.running ? 0 : 1;
        int64_t backlog = 0;
        if (free_slots > 1)
            for (const Request *r : s->pending)
                backlog += r->n;
        for (int k = 0; k < s->nslots && !s->pending.empty(); ++k) {
            if (s->slots[k].running)
                continue;
            const int64_t share =
                free_slots > 1 ? (backlog + free_slots - 1) / free_slots
                               : s->max_batch_pairs;
            std::vector<Request *> take;
            size_t need = 0;
            int64_t pairs = 0;
            while (!s->pending.empty()) {
                Request *r = s->pending.front();
                const bool first = take.empty();
                if (!first && (s->in_use + need + r->footprint > s->budget ||
                               pairs + r->n > s->max_batch_pairs ||
                               pairs >= share))
                    break;
                if (first && s->in_use + r->footprint > s->budget)
                    break;  // wait for memory to free up
                take.push_back(r);
                need += r->footprint;
                pairs += r->n;
                s->pending.pop_front();
            }
            if (take.empty())
                break;
            backlog -= pairs;
            free_slots -= 1;
            const int rc = launch_batch(s, k, take);
            if (rc != SS_OK) {
                for (Request *r : take) {
                    r->state = kDone;
                    r->status = rc;
                    r->t_done = now_s();
                }
                s->sticky_error = rc;
                s->cv_done.notify_all();
                continue;
            }
            s->in_use += s->slots[k].running->bytes;
            int64_t inflight = 0;
            for (Slot &sl : s->slots)
                inflight += sl.running ? 1 : 0;
            s->max_inflight_seen = std::max(s->max_inflight_seen, inflight);
        }
        s->cv_work.wait_for(lock, std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

int ss_server_create(ss_server **out, int device, size_t hbm_budget_bytes,
                     int slots)
{
    if (!out || slots < 1 || slots > 16)
        return SS_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        (void)cudaGetLastError();
        return SS_ERR_CUDA;
    }
    if (device < 0 || device >= ndev)
        return SS_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess)
        return SS_ERR_CUDA;
    auto s = new ss_server();
    s->device = device;
    s->nslots = slots;
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : ((size_t)8 << 30);
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount,
                           device);
    // batch memory from a pool of the server's own, which keeps freed
    // blocks for the next batches (the process's default pool is left as
    // it is)
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    uint64_t keep = UINT64_MAX;
    // the long-pair queue: ring, counters and descriptors on the device;
    // done words and the stop word in host-mapped memory
    const size_t ring_bytes = sizeof(ssk::LongEntry) * ssk::kLongRing;
    const size_t lq_bytes = ring_bytes + 256 +
                            sizeof(ssk::LongBatch) * ssk::kLongBatches;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold,
                                &keep) != cudaSuccess ||
        ssk::bucket_init() != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&s->wst, cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&s->wev, cudaEventDisableTiming) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_long_worker,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)worker_smem()) != cudaSuccess ||
        // an SM holding a worker CTA is set up with all its shared memory,
        // so the batches' kernels still find room beside it (with a
        // smaller split they waited for the worker to leave)
        cudaFuncSetAttribute(k_long_worker,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaMalloc(&s->lq_dev, lq_bytes) != cudaSuccess ||
        cudaMemset(s->lq_dev, 0, lq_bytes) != cudaSuccess ||
        cudaHostAlloc((void **)&s->lq_host,
                      sizeof(int) * (ssk::kLongBatches + 1),
                      cudaHostAllocMapped) != cudaSuccess) {
        (void)cudaGetLastError();
        ss_server_destroy(s);
        return SS_ERR_CUDA;
    }
    std::memset(s->lq_host, 0, sizeof(int) * (ssk::kLongBatches + 1));
    {
        char *q = (char *)s->lq_dev;
        s->lq.ring = (ssk::LongEntry *)q;
        s->lq.tail = (unsigned long long *)(q + ring_bytes);
        s->lq.head = (unsigned long long *)(q + ring_bytes + 8);
        s->lq.last = (unsigned long long *)(q + ring_bytes + 16);
        s->lq.busy = (int *)(q + ring_bytes + 24);
        s->lq.batches = (ssk::LongBatch *)(q + ring_bytes + 256);
        int *hd = nullptr;
        if (cudaHostGetDevicePointer((void **)&hd, s->lq_host, 0) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            ss_server_destroy(s);
            return SS_ERR_CUDA;
        }
        s->lq.done = hd;
        s->lq.stop = hd + ssk::kLongBatches;
        for (int i = ssk::kLongBatches - 1; i >= 0; --i)
            s->lq_free.push_back(i);
    }
    s->slots.resize(slots);
    for (Slot &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) !=
                cudaSuccess ||
            cudaStreamCreateWithFlags(&sl.side, cudaStreamNonBlocking) !=
                cudaSuccess ||
            cudaEventCreateWithFlags(&sl.fork, cudaEventDisableTiming) !=
                cudaSuccess ||
            cudaEventCreateWithFlags(&sl.join, cudaEventDisableTiming) !=
                cudaSuccess) {
            (void)cudaGetLastError();
            ss_server_destroy(s);
            return SS_ERR_CUDA;
        }
    }
    s->thread = std::thread(scheduler, s);
    *out = s;
    return SS_OK;
}

int ss_server_destroy(ss_server *s)
{
    if (!s)
        return SS_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->thread.joinable())
        s->thread.join();
    cudaSetDevice(s->device);
    if (s->lq_host)
        ((volatile int *)s->lq_host)[ssk::kLongBatches] = 1;  // workers leave
    cudaDeviceSynchronize();
    for (auto &b : s->draining) {
        b->pinned_refs = 0;
        maybe_free_batch(s, b);
    }
    for (auto &kv : s->reqs) {
        Request *r = kv.second.get();
        if (r->batch) {
            r->batch->pinned_refs = std::max(0, r->batch->pinned_refs - 1);
            maybe_free_batch(s, r->batch);
            r->batch.reset();
        }
    }
    for (Slot &sl : s->slots) {
        if (sl.running) {
            sl.running->pinned_refs = 0;
            maybe_free_batch(s, sl.running);
        }
        if (sl.st)
            cudaStreamDestroy(sl.st);
        if (sl.side)
            cudaStreamDestroy(sl.side);
        if (sl.fork)
            cudaEventDestroy(sl.fork);
        if (sl.join)
            cudaEventDestroy(sl.join);
    }
    if (s->copy_st)
        cudaStreamDestroy(s->copy_st);
    if (s->wst)
        cudaStreamDestroy(s->wst);
    if (s->wev)
        cudaEventDestroy(s->wev);
    cudaDeviceSynchronize();
    if (s->lq_dev)
        cudaFree(s->lq_dev);
    if (s->lq_host)
        cudaFreeHost(s->lq_host);
    if (s->pool)
        cudaMemPoolDestroy(s->pool);
    (void)cudaGetLastError();
    delete s;
    return SS_OK;
}

int ss_server_submit(ss_server *s, const uint8_t *reads, const uint8_t *refs,
                     const int32_t *lengths, const int32_t *E, int64_t n,
                     uint64_t *ticket)
{
    if (!s || !ticket || n < 1 || n > (1 << 20) || !lengths || !E)
        return SS_ERR_INVALID_ARG;
    auto r = std::make_unique<Request>();
    r->reads = reads;
    r->refs = refs;
    r->n = n;
    r->lengths.assign(lengths, lengths + n);
    r->E.assign(E, E + n);
    r->offsets.resize((size_t)n);
    int64_t bases = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (lengths[k] < 0 || E[k] < 0)
            return SS_ERR_INVALID_ARG;
        r->offsets[(size_t)k] = bases;
        bases += lengths[k];
    }
    if (bases > 0 && (!reads || !refs))
        return SS_ERR_INVALID_ARG;
    r->bases = bases;
    r->footprint = footprint_of(*r);
    std::lock_guard<std::mutex> lock(s->mu);
    if (r->footprint > s->budget)
        return SS_ERR_OOM;
    r->id = s->next_id++;
    r->t_submit = now_s();
    if (s->t_first_submit == 0)
        s->t_first_submit = r->t_submit;
    *ticket = r->id;
    s->pending.push_back(r.get());
    s->reqs.emplace(r->id, std::move(r));
    s->cv_work.notify_one();
    return SS_OK;
}

int ss_server_poll(ss_server *s, uint64_t ticket)
{
    if (!s)
        return SS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return SS_ERR_INVALID_ARG;
    const Request *r = it->second.get();
    if (r->state != kDone)
        return SS_ERR_BUSY;
    return r->status;
}

int ss_server_wait(ss_server *s, uint64_t ticket, int64_t timeout_us)
{
    if (!s)
        return SS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return SS_ERR_INVALID_ARG;
    const Request *r = it->second.get();
    const auto deadline =
        Clock::now() + std::chrono::microseconds(std::max<int64_t>(0, timeout_us));
    while (r->state != kDone) {
        if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout &&
            r->state != kDone)
            return SS_ERR_TIMEOUT;
    }
    return r->status;
}

int ss_server_fetch(ss_server *s, uint64_t ticket, uint8_t *out_accept,
                    int32_t *out_obstacles, double *latency_s)
{
    if (!s || !out_accept || !out_obstacles)
        return SS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return SS_ERR_INVALID_ARG;
    Request *r = it->second.get();
    if (r->state != kDone)
        return SS_ERR_BUSY;
    int rc = r->status;
    if (r->batch && r->batch->dev) {
        cudaSetDevice(s->device);
        if (read_back(s, out_accept, r->batch->acc + r->first,
                      (size_t)r->n) != cudaSuccess ||
            read_back(s, out_obstacles, r->batch->obs + r->first,
                      (size_t)r->n * 4) != cudaSuccess) {
            (void)cudaGetLastError();
            rc = SS_ERR_CUDA;
        }
    } else if (rc == SS_OK) {
        rc = SS_ERR_CUDA;
    }
    if (latency_s)
        *latency_s = r->t_done - r->t_submit;
    if (r->batch) {
        r->batch->pinned_refs -= 1;
        maybe_free_batch(s, r->batch);
        r->batch.reset();
    }
    s->reqs.erase(it);
    s->cv_work.notify_one();
    return rc;
}

int ss_server_get_stats(ss_server *s, ss_server_stats *out)
{
    if (!s || !out)
        return SS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    std::memset(out, 0, sizeof *out);
    out->requests_done = s->done_requests;
    out->pairs_done = s->done_pairs;
    out->bases_done = s->done_bases;
    out->batches = s->batches;
    out->max_inflight = s->max_inflight_seen;
    out->pending = (int64_t)s->pending.size();
    out->device_bytes_in_use = (int64_t)s->in_use;
    out->long_pairs_queued = s->long_queued;
    out->worker_launches = s->worker_launches;
    std::vector<double> v = s->latencies;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const size_t i = (size_t)std::min<double>(
                (double)(v.size() - 1), q * (double)(v.size() - 1) + 0.5);
            return v[i];
        };
        out->latency_p50_s = pct(0.50);
        out->latency_p99_s = pct(0.99);
        out->latency_max_s = v.back();
    }
    if (s->t_last_done > s->t_first_submit && s->t_first_submit > 0)
        out->span_s = s->t_last_done - s->t_first_submit;
    return s->sticky_error;
}

int ss_server_reset_stats(ss_server *s)
{
    if (!s)
        return SS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    s->latencies.clear();
    s->done_requests = s->done_pairs = s->done_bases = 0;
    s->batches = s->max_inflight_seen = 0;
    s->long_queued = s->worker_launches = 0;
    s->t_first_submit = s->t_last_done = 0;
    s->sticky_error = SS_OK;
    return SS_OK;
}

}  // extern "C"
