/*
 * ss.h -- C ABI of the SneakySnake pre-alignment filter for GB300 (sm_103a).
 *
 * What it computes (Alser et al., "SneakySnake", Section 2.3-2.4): for each
 * pair of a reference segment R[1..m] and a query (read) Q[1..m] and an edit
 * threshold E, the chip maze Z of Eq. 1 -- 2E+1 rows (HRTs) x m columns
 * (VRTs), Z[i,j] = 0 where R[j] equals the Q base on diagonal i, else 1 --
 * and the greedy single-net-routing solution of Section 2.4: from checkpoint
 * column 1, repeatedly take the longest run of zeros over all rows, count the
 * obstacle that ends it, and move the checkpoint past it; stop at the row end
 * or once the count exceeds E.  Per pair the library returns
 *     accept    = (count <= E)                (1 byte: 1 = alignment needed)
 *     obstacles = min(count, E + 1)           (int32)
 * Results are bit-identical to a plain CPU reading of the paper.
 *
 * Memory: every data pointer is a DEVICE pointer owned by the caller, except
 * in ss_filter_host(), which takes host pointers.  The library allocates
 * only its own workspace, inside the context, within the budget given to
 * ss_create().  Calls are asynchronous on the given CUDA stream (a
 * cudaStream_t; NULL = the CUDA default stream) and return a launch-time
 * status; errors found by the
 * kernels (a non-ACGT byte, a negative per-pair length or threshold) are
 * latched in the context and returned by ss_sync().
 *
 * Threading: a context may be used by one host thread at a time; contexts
 * (and servers) may be created and used from several host threads at once,
 * on one device or several.
 */
#ifndef SS_H
#define SS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SS_OK 0
#define SS_ERR_INVALID_ARG (-1)  /* bad scalar/pointer, or bad per-pair value */
#define SS_ERR_INVALID_BASE (-2) /* an input byte is not A/C/G/T (any case)  */
#define SS_ERR_OOM (-3)          /* workspace would exceed the budget         */
#define SS_ERR_CUDA (-4)         /* a CUDA runtime call failed                */
#define SS_ERR_TIMEOUT (-5)      /* a bounded device-side wait gave up        */
#define SS_ERR_BUSY (-6)         /* no free slot (serving admission)          */
#define SS_ERR_UNSUPPORTED (-7)  /* shape outside what the build supports     */

/* ---- input formats -------------------------------------------------------
 * SS_FMT_ASCII   : one byte per base, 'A','C','G','T' in either case.
 * SS_FMT_PACKED2 : 2 bits per base, 16 bases per little-endian uint32 word.
 *   Base j of a sequence lives in word j/16: bit (j%16) holds bit 0 of its
 *   code and bit 16+(j%16) holds bit 1, with codes A=0, C=1, G=2, T=3.  A
 *   sequence of m bases takes ss_packed_words(m) = ceil(m/16) words; unused
 *   bits are zero.  ss_pack() writes this format.                          */
#define SS_FMT_ASCII 0
#define SS_FMT_PACKED2 1
/* SS_FMT_SLICED2 : 2 bits per base, bit-sliced over groups of 32 pairs,
 *   for fixed-stride batches (every pair of length m).  Pair p is bit p%32
 *   of group g = p/32 (G = ceil(n/32) groups).  Bit b (0 or 1) of the code
 *   of base j of the group's 32 sequences is one uint32 word, at index
 *       ((j/4 * G + g) * 2 + b) * 4 + j%4
 *   so four consecutive bases of one code bit are 16 contiguous bytes.
 *   One side (reads or refs) of n pairs takes ss_sliced_words(m, n) =
 *   8 * ceil(m/4) * G words (2 bits per base, 25 bytes per pair at m =
 *   100); bits of pairs p >= n and words of bases j >= m are zero.
 *   ss_pack_sliced() writes this format.  The filter walks the 32 pairs of
 *   a group at once, one pair per bit. */
#define SS_FMT_SLICED2 2

/* ---- filter modes (flags of ss_filter_batch) -------------------------- */
#define SS_MODE_AUTO 0     /* plain launch if m and E are uniform, else bucketed */
#define SS_MODE_PLAIN 1    /* one launch per (m, E) group, no queue            */
#define SS_MODE_BUCKETED 2 /* length/threshold-bucketed persistent launch      */
#define SS_FLAG_NO_GRAPH 16 /* do not replay the captured CUDA graph           */

/* Largest E of the plain launch over SS_FMT_SLICED2 input. */
#define SS_SLICED_MAX_E 31

/* Largest uniform E and m the plain launch covers. */
#define SS_PLAIN_MAX_E 31
#define SS_PLAIN_MAX_M 1024

typedef struct ss_ctx ss_ctx;

/* Create a context on CUDA device `device` with a workspace budget of
 * `workspace_bytes` (0 = 1 GiB).  The context owns one CUDA stream and a
 * small device status word; the stream orders internal work only (calls run
 * on the stream the caller passes).  Returns SS_OK, SS_ERR_INVALID_ARG (out NULL or
 * bad device) or SS_ERR_CUDA. */
int ss_create(ss_ctx **out, int device, size_t workspace_bytes);

/* Release everything the context owns.  NULL is accepted. */
int ss_destroy(ss_ctx *ctx);

/* Human-readable text of a status code (static storage). */
const char *ss_strerror(int code);

/* ABI version (major * 10000 + minor * 100 + patch). */
int ss_version(void);

/* Words of the packed format needed for m bases: ceil(m / 16). */
int64_t ss_packed_words(int64_t m);

/* Pack n ASCII sequences into the SS_FMT_PACKED2 format (step Eq. 1 needs
 * only base equality, so any fixed code works; this one is documented above).
 *   ascii          device; sequence p starts at byte offsets[p] (or p*m when
 *                  offsets is NULL) and has lengths[p] (or m) bases.
 *   packed         device, output; sequence p starts at word
 *                  packed_offsets[p] (or p*ceil(m/16) when NULL).
 * A non-ACGT byte latches SS_ERR_INVALID_BASE (returned by ss_sync); the
 * affected words are written with that byte's code taken as A.
 * offsets/lengths/packed_offsets must be all NULL (fixed stride) or all
 * non-NULL.  Returns SS_OK, SS_ERR_INVALID_ARG or SS_ERR_CUDA. */
int ss_pack(ss_ctx *ctx, const uint8_t *ascii, const int64_t *offsets,
            const int32_t *lengths, int32_t m, int64_t n, uint32_t *packed,
            const int64_t *packed_offsets, void *stream);

/* Words of the SS_FMT_SLICED2 format for n sequences of m bases:
 * 8 * ceil(m/4) * ceil(n/32) (0 if n or m is not positive). */
int64_t ss_sliced_words(int64_t m, int64_t n);

/* Pack n fixed-stride ASCII sequences of m bases (sequence p at ascii +
 * p*m, device) into the SS_FMT_SLICED2 format at `sliced` (device,
 * ss_sliced_words(m, n) words, 16-byte aligned).  Every word of the output
 * is written.  A non-ACGT byte latches SS_ERR_INVALID_BASE (returned by
 * ss_sync), its code taken as A.  Returns SS_OK, SS_ERR_INVALID_ARG or
 * SS_ERR_CUDA. */
int ss_pack_sliced(ss_ctx *ctx, const uint8_t *ascii, int32_t m, int64_t n,
                   uint32_t *sliced, void *stream);

/* Filter n equal-length read/reference pairs (Section 2.4).
 *   reads, refs    device; format SS_FMT_ASCII, SS_FMT_PACKED2 or
 *                  SS_FMT_SLICED2 (the last with a fixed stride, uniform m,
 *                  scalar e <= SS_SLICED_MAX_E, 16-byte aligned reads,
 *                  refs; SS_ERR_UNSUPPORTED for a larger e or
 *                  SS_MODE_BUCKETED).  Pair p's
 *                  query is reads + offsets[p] and its reference is
 *                  refs + offsets[p] (units: bytes for ASCII, 32-bit words
 *                  for PACKED2).  offsets == NULL means a fixed stride of m
 *                  bases per pair (m bytes, or ceil(m/16) words).
 *   lengths        device int32[n] per-pair m (>= 0), or NULL with scalar m.
 *   E              device int32[n] per-pair threshold (>= 0), or NULL with
 *                  scalar e.
 *   n              number of pairs (>= 0; 0 is a no-op).
 *   flags          SS_MODE_* | SS_FLAG_*.
 *   out_accept     device uint8[n]: 1 if count <= E (alignment needed).
 *   out_obstacles  device int32[n]: min(count, E+1); -1 for a pair with a
 *                  negative length or threshold (which also latches
 *                  SS_ERR_INVALID_ARG).
 * With offsets != NULL, lengths must be non-NULL.  ASCII input must have a
 * fixed stride (per-pair offsets need PACKED2: pack first with ss_pack); it
 * is packed into context workspace chunk by chunk (SS_ERR_OOM if one pair
 * does not fit the budget).  Per-pair lengths up to 131072 are supported
 * for any E (longer pairs with E' > 31 latch SS_ERR_UNSUPPORTED and get
 * obstacles = -1).  Calls that use the workspace (ASCII input, the bucketed
 * form) must not overlap on the GPU for one context.
 * Returns SS_OK, SS_ERR_INVALID_ARG, SS_ERR_OOM, SS_ERR_UNSUPPORTED (MODE_PLAIN
 * on a shape the plain kernel does not cover) or SS_ERR_CUDA. */
int ss_filter_batch(ss_ctx *ctx, const void *reads, const void *refs,
                    int format, const int64_t *offsets,
                    const int32_t *lengths, int32_t m, const int32_t *E,
                    int32_t e, int64_t n, int flags, void *stream,
                    uint8_t *out_accept, int32_t *out_obstacles);

/* A threshold sweep on the device: n fixed-stride pairs of uniform length m
 * (device, format SS_FMT_ASCII, SS_FMT_PACKED2 or SS_FMT_SLICED2 -- the last
 * 16-byte aligned) filtered at each of the n_e thresholds of the host array
 * e_list.  Outputs are DEVICE arrays laid out [n_e][n]: out_accept[t * n +
 * p], out_obstacles[t * n + p].  Over the sliced layout (ASCII input with
 * every threshold up to SS_SLICED_MAX_E is packed to it, chunk by chunk in
 * the context's workspace), the distinct thresholds from 0 to 4 share one
 * pass over the pairs (their walks cost less than reading the pairs) and
 * every other threshold gets its own launch; PACKED2 input is filtered one
 * threshold at a time.  Returns SS_OK, SS_ERR_INVALID_ARG, SS_ERR_OOM,
 * SS_ERR_UNSUPPORTED (sliced input with a threshold above SS_SLICED_MAX_E)
 * or SS_ERR_CUDA; device-side errors through ss_sync. */
int ss_filter_sweep(ss_ctx *ctx, const void *reads, const void *refs,
                    int format, int32_t m, const int32_t *e_list, int n_e,
                    int64_t n, void *stream, uint8_t *out_accept,
                    int32_t *out_obstacles);

/* One batch of a segmented call: n fixed-stride pairs, reads of m bases
 * against references of m_ref bases (0: m, equal lengths), filtered at
 * threshold e (Section 2.4), in the call's format.  When m_ref differs
 * from m, the maze has one column per reference base and the cells where a
 * diagonal reads no base of the read are free, not obstacles (Section
 * 2.4's correction of the leading and trailing obstacles). */
typedef struct ss_segment {
    const void *reads;       /* device; SS_FMT_SLICED2: 16-byte aligned      */
    const void *refs;        /* device; same layout as reads, m_ref bases    */
    int64_t n;               /* pairs (>= 0; 0: the segment is skipped)      */
    int32_t m;               /* bases per read (>= 0)                        */
    int32_t e;               /* threshold (>= 0)                             */
    uint8_t *out_accept;     /* device uint8[n]: 1 if count <= e             */
    int32_t *out_obstacles;  /* device int32[n]: min(count, e + 1)           */
    int32_t m_ref;           /* bases per reference (>= 0; 0: m)             */
} ss_segment;

/* Several uniform batches (segments, e.g. reads of 150 and of 250 bases,
 * each with its own threshold) filtered by one call: a batch mixing lengths
 * and thresholds, bucketed by the caller into uniform segments.  format is
 * SS_FMT_SLICED2 (every e <= SS_SLICED_MAX_E; reads and references each in
 * the layout of their own length) or SS_FMT_PACKED2 (fixed stride
 * ceil(m/16) words per sequence; equal lengths, m <= SS_PLAIN_MAX_M and e
 * <= SS_PLAIN_MAX_E).  Every segment's launch is independent of the others:
 * they run side by side on the context's streams, the costliest first, so
 * that the GPU does not drain between them; over SS_FMT_SLICED2, segments
 * of one threshold share a launch (up to 32 per launch).  Unless flags holds
 * SS_FLAG_NO_GRAPH, the launches are captured once per distinct segment
 * table (pointers and sizes) as a CUDA graph and replayed.  The segments'
 * outputs must not overlap one another.  The whole table is checked before
 * anything is launched.  Returns SS_OK, SS_ERR_INVALID_ARG, SS_ERR_UNSUPPORTED
 * (a threshold or length the format's kernel does not take) or SS_ERR_CUDA;
 * device-side errors through ss_sync. */
int ss_filter_segments(ss_ctx *ctx, const ss_segment *segs, int n_seg,
                       int format, int flags, void *stream);

/* Fixed-stride pairs of uniform length m held in HOST memory, filtered at
 * each of the n_e thresholds of the host array e_list (a threshold sweep as
 * in Section 3.2 needs the pairs copied once).  The library streams chunks
 * host -> device, packs them (ASCII), runs one plain filter launch per
 * threshold and copies the results back, overlapping copies and compute on
 * two internal streams.  Outputs are HOST arrays laid out [n_e][n]:
 * out_accept[t * n + p], out_obstacles[t * n + p].  Synchronous: returns
 * when the host outputs are written (device errors included).  Pinned host
 * buffers give the full copy bandwidth. */
int ss_filter_host(ss_ctx *ctx, const void *reads, const void *refs,
                   int format, int32_t m, const int32_t *e_list, int n_e,
                   int64_t n, uint8_t *out_accept, int32_t *out_obstacles);

/* Wait for all work on `stream` (NULL = default stream) and for the
 * context's internal streams, and return the first
 * device-side error latched since the previous ss_sync, or SS_OK.  The
 * status word is read and cleared in one atomic exchange: an error latched
 * meanwhile by a launch still running on some other stream is not lost but
 * returned by a later ss_sync. */
int ss_sync(ss_ctx *ctx, void *stream);

/* Self-test of the device-side failure path (not in the paper): launch one
 * kernel that waits on an mbarrier nothing completes, with the same bounded
 * wait the filter kernels use for their bulk copies (which give up after
 * 2 s).  The wait gives up after limit_ns (1e3..1e10) and latches the
 * timeout status, so the next ss_sync on `stream` returns SS_ERR_TIMEOUT and
 * the context stays usable.  Returns SS_OK once launched, SS_ERR_INVALID_ARG
 * or SS_ERR_CUDA. */
int ss_check_wait_timeout(ss_ctx *ctx, int64_t limit_ns, void *stream);

/* ---- batch scheduling of mixed batches (not in the paper: its GPU
 * version runs one thread per pair, Section 2.6) --------------------------
 * A batch with per-pair lengths or thresholds (or E > SS_PLAIN_MAX_E, or
 * m > SS_PLAIN_MAX_M) is filtered in the bucketed form.  Its first kernel
 * walks the batch in tiles of 128 consecutive pairs: a tile whose pairs
 * share one m <= 256 and one E <= SS_PLAIN_MAX_E and lie back to back
 * (pair p + 1's words right after pair p's) is routed at once, as the
 * plain launch routes it.  Every other pair is classified by (m, E') with
 * E' = min(E, m-1), grouped by class and length (longest first), and one
 * persistent kernel per class routes its pairs from an atomic work queue.
 * The whole sequence is captured once in a CUDA graph and replayed for
 * identical arguments; in the graph a class kernel runs only when its
 * class has pairs.  Two knobs change speed, never results:
 *   rw_max_e   15 or 31: largest E' routed with one thread per pair (above
 *              it, one warp or one CTA per pair, rows across the lanes);
 *   cw_subgrid 4, 8 or 16: columns evaluated across all rows per step by
 *              the warp/CTA kernels before surviving runs are extended
 *              32 columns at a time.
 * ss_autotune() times every combination on the given batch (device
 * pointers as in ss_filter_batch, outputs written) and keeps the fastest in
 * the context; ss_set_tuning()/ss_get_tuning() set or read them directly.
 * Returns SS_OK, SS_ERR_INVALID_ARG, SS_ERR_OOM or SS_ERR_CUDA; best_ms
 * (may be NULL) receives the best time per pass. */
int ss_set_tuning(ss_ctx *ctx, int rw_max_e, int cw_subgrid);
int ss_get_tuning(const ss_ctx *ctx, int *rw_max_e, int *cw_subgrid);
int ss_autotune(ss_ctx *ctx, const void *reads, const void *refs,
                const int64_t *offsets, const int32_t *lengths, int32_t m,
                const int32_t *E, int32_t e, int64_t n, void *stream,
                uint8_t *out_accept, int32_t *out_obstacles, int reps,
                float *best_ms);

/* ---- accuracy harness (Section 3.2: false accept / false reject rates
 * against an aligner's ground truth) ----------------------------------------
 * ss_edit_distance_banded: for n fixed-stride SS_FMT_PACKED2 pairs of length
 * m, writes out_ed[p] = min(ED(Q_p, R_p), e + 1) (device int32[n]), the exact
 * Levenshtein distance whenever it is <= e (banded DP over the 2e+1
 * diagonals; any alignment of cost <= e stays inside them).  e <= 31, else
 * SS_ERR_UNSUPPORTED.
 * ss_filter_confusion: out_counts (device uint64[4]) receives, over n pairs
 * with filter decisions accept[] and capped distances ed[] at threshold e:
 * [0] accepted & ED <= e (true accepts), [1] accepted & ED > e (false
 * accepts), [2] rejected & ED <= e (false rejects; 0 for a lossless filter),
 * [3] rejected & ED > e (true rejects).  Both are asynchronous on `stream`.
 * Return SS_OK, SS_ERR_INVALID_ARG, SS_ERR_UNSUPPORTED or SS_ERR_CUDA. */
int ss_edit_distance_banded(ss_ctx *ctx, const void *reads, const void *refs,
                            int format, int32_t m, int32_t e, int64_t n,
                            void *stream, int32_t *out_ed);
int ss_filter_confusion(ss_ctx *ctx, const uint8_t *accept,
                        const int32_t *ed, int64_t n, int32_t e,
                        void *stream, uint64_t *out_counts);
/* ss_edit_distance_varlen: the same capped distance for pairs of per-pair
 * length lengths[p] (both sequences) at word offset offsets[p] of `reads`
 * and `refs` (SS_FMT_PACKED2, int64 word offsets, device arrays) and
 * per-pair threshold E[p] <= 511; one warp per pair, the band spread over
 * its lanes.  out_ed[p] = min(ED, E[p] + 1); a pair with E[p] > 511 gets -1
 * and SS_ERR_UNSUPPORTED from the next ss_sync, a negative length or
 * threshold -1 and SS_ERR_INVALID_ARG.  Asynchronous on `stream`.  Returns
 * SS_OK, SS_ERR_INVALID_ARG or SS_ERR_CUDA. */
int ss_edit_distance_varlen(ss_ctx *ctx, const void *reads, const void *refs,
                            const int64_t *offsets, const int32_t *lengths,
                            const int32_t *E, int64_t n, void *stream,
                            int32_t *out_ed);

/* ---- pairs of different lengths (Section 2.4) ------------------------------
 * Pair p: query (read) of read_len[p] bases at word read_off[p] of `reads`,
 * reference of ref_len[p] bases at word ref_off[p] of `refs` (both
 * SS_FMT_PACKED2, int64 word offsets, int32 lengths, device arrays),
 * threshold E[p] (E = NULL: e for every pair).  The maze has ref_len[p]
 * columns (Eq. 1 compares the reference base of each column with 2E+1 query
 * bases).  With equal lengths the pair is filtered as by ss_filter_batch.
 * When the lengths differ, the leading and trailing obstacles that case 4 of
 * Eq. 1 causes -- cells whose query index falls before the query's first
 * base or after its last -- are deducted, read as: those cells are not
 * obstacles, so overhanging ends of either sequence cost nothing.  The
 * count then never exceeds the edit distance of the query to the stretch of
 * the reference it overlaps (no false reject for approximate string
 * matching), and the greedy still finds the fewest obstacles (Theorem 2).
 * Rows: min(E, m - 1) for equal lengths m; with different lengths E, or 0
 * obstacles outright when E >= min(read_len, ref_len) (a diagonal that
 * compares nothing).  More than 31 rows: obstacles -1, accept 0 and
 * SS_ERR_UNSUPPORTED from the next ss_sync; a negative length or threshold:
 * -1 and SS_ERR_INVALID_ARG.  Asynchronous on `stream`.  Returns SS_OK,
 * SS_ERR_INVALID_ARG or SS_ERR_CUDA. */
int ss_filter_unequal(ss_ctx *ctx, const void *reads, const int64_t *read_off,
                      const int32_t *read_len, const void *refs,
                      const int64_t *ref_off, const int32_t *ref_len,
                      const int32_t *E, int32_t e, int64_t n, void *stream,
                      uint8_t *out_accept, int32_t *out_obstacles);

/* ---- sub-maze approximate mode (Section 2.5, Snake-on-Chip) -------------
 * The maze is cut into sub-mazes of t consecutive columns (the last may be
 * narrower); each is routed independently by the greedy of Section 2.4 from
 * its first column to its last, counting at most y escape segments (the
 * reading taken of the paper's "y module instances per sub-maze"); the
 * counts are summed and capped at e+1.  accept = (sum <= e).  The paper
 * notes that this can only underestimate the exact count (more false
 * accepts, never a false reject); t >= m with y > e gives the exact filter.
 * Fixed-stride SS_FMT_PACKED2 pairs of length m with min(e, m-1) <= 31, or
 * SS_FMT_SLICED2 pairs (16-byte aligned) with e <= SS_SLICED_MAX_E, walked
 * 32 pairs per thread (else SS_ERR_UNSUPPORTED); t, y >= 1.  For m <= 256 the pairs are staged by
 * bulk copies whose bounded waits, should one give up, latch SS_ERR_TIMEOUT
 * for the next ss_sync.  Asynchronous on `stream`.  Returns SS_OK,
 * SS_ERR_INVALID_ARG, SS_ERR_UNSUPPORTED or SS_ERR_CUDA. */
int ss_filter_submaze(ss_ctx *ctx, const void *reads, const void *refs,
                      int format, int32_t m, int32_t e, int32_t t, int32_t y,
                      int64_t n, void *stream, uint8_t *out_accept,
                      int32_t *out_obstacles);

/* ---- downstream pass-through: the accepted pairs (Section 2.4 step 5,
 * "sequence alignment is needed") for an aligner ------------------------------
 * ss_compact_accepted: out_index (device int64[n]) receives, in increasing
 * order, the indices p with accept[p] != 0; *out_count (device int64) their
 * number.  Uses context workspace (8 bytes per 4096 pairs); asynchronous.
 * ss_gather_pairs: for fixed-stride SS_FMT_PACKED2 pairs of length m, copies
 * pair index[i] of reads/refs to slot i of out_reads/out_refs for every
 * i < min(*count, n) (device count, so it can follow ss_compact_accepted
 * without a host round trip); reads/refs hold n pairs and out_reads/out_refs
 * n slots of ceil(m/16) words; indices outside 0..n-1 are skipped.  Both
 * return SS_OK,
 * SS_ERR_INVALID_ARG, SS_ERR_OOM or SS_ERR_CUDA. */
int ss_compact_accepted(ss_ctx *ctx, const uint8_t *accept, int64_t n,
                        void *stream, int64_t *out_index, int64_t *out_count);
int ss_gather_pairs(ss_ctx *ctx, const void *reads, const void *refs,
                    int32_t m, const int64_t *index, const int64_t *count,
                    int64_t n, void *stream, void *out_reads,
                    void *out_refs);

/* ---- allocation-free entry point (the paper has no counterpart) -------
 * For callers that cannot allocate device memory: a service that reserves
 * all of a GPU's memory up front through its own allocator (an extra
 * cudaMalloc would fail, or would synchronise the device at an unpredictable
 * moment), or a plug-in inside another program that must stay within that
 * program's memory.  Same arguments and results as ss_filter_batch for
 * SS_FMT_PACKED2 input in the bucketed form (default tuning), but with no
 * context and no allocation: the scratch (class tables and the pair
 * permutation) is one fixed __device__ array of about 4 MiB in the library,
 * held by every GPU that loads it until the process exits.
 *   - Runs on the CURRENT device, on `stream` (NULL = default stream).  The
 *     first call on a device looks up the array's device address and sizes
 *     the kernels' grids; make that first call before any stream capture.
 *   - n must be <= SS_NOALLOC_MAX_PAIRS, else SS_ERR_OOM (nothing launched).
 *   - All calls share the one array and it keeps the last call's contents:
 *     calls that overlap on the GPU (other streams or host threads) race.
 *     Order them on one stream or synchronise between them.
 *   - There is no ss_sync for it and no status is reported: a pair with a
 *     negative length or threshold, or one longer than 131072 bases (too
 *     long to stage), gets obstacles = -1 and accept = 0; the kernels'
 *     status flags go to a word of the scratch array that nothing reads.
 * Returns SS_OK, SS_ERR_INVALID_ARG, SS_ERR_OOM or SS_ERR_CUDA. */
#define SS_NOALLOC_MAX_PAIRS 1048576
int ss_filter_batch_noalloc(const void *reads, const void *refs,
                            const int64_t *offsets, const int32_t *lengths,
                            int32_t m, const int32_t *E, int32_t e, int64_t n,
                            void *stream, uint8_t *out_accept,
                            int32_t *out_obstacles);

/* ---- serving: continuous batching of filter requests (not in the paper;
 * its GPU version filters one prepared batch) -------------------------------
 * A server owns a scheduler thread and `slots` in-flight batch slots.  A
 * request is n pairs in HOST memory: ASCII reads and refs concatenated
 * (pair k at byte sum(lengths[0..k-1])), per-pair lengths and thresholds.
 * Whenever a slot is free the scheduler admits pending requests first-in
 * first-out while their device footprint fits `hbm_budget_bytes`, copies
 * them to the device, packs them and runs the bucketed filter with its
 * persistent grids sized to 1/slots of the SMs, so batches admitted while
 * others run execute beside them.  Results stay in device memory until
 * fetched, and a batch's device memory counts against the budget until all
 * of its requests are fetched: a client that waits for later requests
 * before fetching earlier ones can fill the budget and stall admission, so
 * fetch each result once it is done.  A request whose bases are not all
 * A/C/G/T fails alone
 * (SS_ERR_INVALID_BASE; its bad pairs get obstacles = -1).
 *   ss_server_create   device, budget (0 = 8 GiB), slots 1..16.
 *   ss_server_submit   1 <= n <= 2^20; the host buffers must stay valid and
 *                      unchanged until the request is done (pinned memory
 *                      copies fastest).  Returns SS_ERR_OOM if the request
 *                      alone exceeds the budget.  *ticket identifies it.
 *   ss_server_poll     SS_ERR_BUSY while pending/running, else its status.
 *   ss_server_wait     blocks up to timeout_us; SS_ERR_TIMEOUT if not done.
 *   ss_server_fetch    copies the results to host arrays of n entries,
 *                      frees the request; latency_s (may be NULL) receives
 *                      completion minus submission time.
 *   ss_server_get_stats / ss_server_reset_stats  latency percentiles of the
 *                      completed requests and counters.
 * A server is driven from any number of client threads. */
typedef struct ss_server ss_server;
typedef struct ss_server_stats {
    int64_t requests_done, pairs_done, bases_done;
    int64_t batches;        /* batches launched                         */
    int64_t max_inflight;   /* most batches seen in flight at once       */
    int64_t pending;        /* requests waiting for admission            */
    int64_t device_bytes_in_use;
    double latency_p50_s, latency_p99_s, latency_max_s;
    double span_s;          /* first submission to last completion       */
    int64_t long_pairs_queued; /* pairs routed by the long-pair queue    */
    int64_t worker_launches;   /* launches of its long-lived worker      */
} ss_server_stats;
int ss_server_create(ss_server **out, int device, size_t hbm_budget_bytes,
                     int slots);
int ss_server_submit(ss_server *srv, const uint8_t *reads,
                     const uint8_t *refs, const int32_t *lengths,
                     const int32_t *E, int64_t n, uint64_t *ticket);
int ss_server_poll(ss_server *srv, uint64_t ticket);
int ss_server_wait(ss_server *srv, uint64_t ticket, int64_t timeout_us);
int ss_server_fetch(ss_server *srv, uint64_t ticket, uint8_t *out_accept,
                    int32_t *out_obstacles, double *latency_s);
int ss_server_get_stats(ss_server *srv, ss_server_stats *out);
int ss_server_reset_stats(ss_server *srv);
int ss_server_destroy(ss_server *srv);

/* Counters of the context since creation (host-side accounting). */
typedef struct ss_counters {
    int64_t pairs;        /* pairs submitted to ss_filter_batch/_host */
    int64_t launches;     /* kernels launched by the library          */
    int64_t graph_replays;/* CUDA graph launches                      */
    int64_t workspace_bytes; /* device workspace currently held       */
} ss_counters;
int ss_get_counters(const ss_ctx *ctx, ss_counters *out);

#ifdef __cplusplus
}
#endif
#endif
