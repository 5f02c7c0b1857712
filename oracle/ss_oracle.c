/*
 * ss_oracle.c -- plain CPU SneakySnake, written from the paper's definition.
 *
 * TEST INFRASTRUCTURE ONLY (see ss_oracle.h).  Deliberately slow and literal:
 * every maze entry is evaluated through Eq. 1 one at a time, with 1-based
 * indices as in the paper, and the greedy routing follows the five steps of
 * Section 2.4 in order.  Independent pairs are spread over host threads; that
 * is the only departure from a single loop and it changes no arithmetic.
 *
 * Readings of the paper taken here (where it is silent or loose):
 *  - An entry whose Q index falls outside 1..m is an obstacle (Eq. 1, the
 *    "otherwise" case).
 *  - A run of zeros that reaches column m ends the routing with no obstacle
 *    counted (Section 2.4 step 2: a segment ends at an obstacle or at the end
 *    of the row; an escape segment holds at most one obstacle, Section 2.2).
 *  - The count stops growing once it exceeds E (step 4), so the reported
 *    obstacle count is min(count, E+1); accept iff count <= E (step 5).
 *  - Bases compare case-insensitively; any byte other than A/C/G/T is an
 *    error (the paper does not define other symbols).
 *  - Only equal-length pairs (|Q| = |R| = m), the paper's simplifying case in
 *    Section 2.3.  m = 0 is allowed: nothing to route, count 0, accept.
 */
#include "ss_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* Canonical base of a byte, or 0 if it is not a nucleotide. */
static int base_of(uint8_t c)
{
    switch (c) {
    case 'A': case 'a': return 'A';
    case 'C': case 'c': return 'C';
    case 'G': case 'g': return 'G';
    case 'T': case 't': return 'T';
    default: return 0;
    }
}

/* Two symbols are equal if they are the same base (in any case) or the
 * same byte. */
static int same_symbol(uint8_t a, uint8_t b)
{
    return a == b || (base_of(a) != 0 && base_of(a) == base_of(b));
}

static int valid_sequence(const uint8_t *s, int64_t m)
{
    for (int64_t k = 0; k < m; ++k)
        if (!base_of(s[k]))
            return 0;
    return 1;
}

/* Eq. 1.  Row i = E+1 compares Q[j] with R[j] (case 1); rows 1..E compare
 * Q[j-i] (case 2, the E left-hand neighbours, deletions in Q); rows
 * E+2..2E+1 compare Q[j+i-E-1] (case 3, right-hand neighbours, insertions
 * in Q); everything else is an obstacle (case 4). */
int sso_cell(const uint8_t *Q, const uint8_t *R, int64_t m, int64_t E,
             int64_t i, int64_t j)
{
    int64_t q;
    if (i == E + 1)
        q = j;
    else if (i >= 1 && i <= E)
        q = j - i;
    else
        q = j + i - E - 1;
    if (q < 1 || q > m)
        return 1;
    return base_of(Q[q - 1]) == base_of(R[j - 1]) ? 0 : 1;
}

int sso_maze(const uint8_t *Q, const uint8_t *R, int64_t m, int64_t E,
             uint8_t *Z)
{
    if (m < 0 || E < 0)
        return SSO_ERR_INVALID_ARG;
    if (!valid_sequence(Q, m) || !valid_sequence(R, m))
        return SSO_ERR_INVALID_BASE;
    for (int64_t i = 1; i <= 2 * E + 1; ++i)
        for (int64_t j = 1; j <= m; ++j)
            Z[(i - 1) * m + (j - 1)] = (uint8_t)sso_cell(Q, R, m, E, i, j);
    return SSO_OK;
}

/* Step (2) for one row: length of the first horizontal run of zeros that
 * starts at the checkpoint and ends at an obstacle or at the end of the row.
 * Counts the entries it had to evaluate (the implicit maze of Section 2.4). */
static int64_t run_from_checkpoint(const uint8_t *Q, const uint8_t *R,
                                   int64_t m, int64_t E, int64_t i,
                                   int64_t checkpoint, int64_t *evaluated)
{
    int64_t len = 0;
    int64_t seen = 0;
    for (int64_t j = checkpoint; j <= m; ++j) {
        ++seen;
        if (sso_cell(Q, R, m, E, i, j) != 0)
            break;
        ++len;
    }
    *evaluated = seen;
    return len;
}

int sso_filter(const uint8_t *Q, const uint8_t *R, int64_t m, int64_t E,
               int stop_above_E, uint8_t *accept, int64_t *obstacles,
               sso_stats *stats)
{
    if (m < 0 || E < 0)
        return SSO_ERR_INVALID_ARG;
    if (!valid_sequence(Q, m) || !valid_sequence(R, m))
        return SSO_ERR_INVALID_BASE;

    sso_stats st = {0, 0, 0, 0};
    /* Step (1): the maze is implicit; the first column is the first
     * checkpoint. */
    int64_t checkpoint = 1;
    int64_t count = 0; /* obstacles on the signal net so far */

    while (checkpoint <= m) {
        /* Step (2): the longest of the 2E+1 horizontal segments. */
        int64_t longest = 0;
        st.iterations += 1;
        for (int64_t i = 1; i <= 2 * E + 1; ++i) {
            int64_t evaluated = 0;
            int64_t len =
                run_from_checkpoint(Q, R, m, E, i, checkpoint, &evaluated);
            st.cells += evaluated;
            st.words += (evaluated + 31) / 32;
            if (len > longest)
                longest = len;
        }
        /* The segment reaches the end of the row: the signal net has reached
         * the destination terminal, no obstacle follows it. */
        if (checkpoint + longest > m) {
            st.columns += m - checkpoint + 1;
            break;
        }
        st.columns += longest + 1;
        /* Otherwise the escape segment is the run plus the obstacle that
         * follows it (a lone obstacle when longest = 0). */
        count += 1;
        /* Step (3): new checkpoint right after the escape segment. */
        checkpoint = checkpoint + longest + 1;
        /* Step (4): stop once the delay exceeds E x t_obstacle. */
        if (stop_above_E && count > E)
            break;
    }
    /* Step (5). */
    if (accept)
        *accept = (uint8_t)(count <= E);
    if (obstacles)
        *obstacles = count;
    if (stats)
        *stats = st;
    return SSO_OK;
}

int sso_filter_submaze(const uint8_t *Q, const uint8_t *R, int64_t m,
                       int64_t E, int64_t t, int64_t y, uint8_t *accept,
                       int64_t *obstacles)
{
    if (m < 0 || E < 0 || t < 1 || y < 1)
        return SSO_ERR_INVALID_ARG;
    if (!valid_sequence(Q, m) || !valid_sequence(R, m))
        return SSO_ERR_INVALID_BASE;
    int64_t count = 0;
    for (int64_t first = 1; first <= m && count <= E; first += t) {
        const int64_t last = first + t - 1 < m ? first + t - 1 : m;
        /* the greedy of Section 2.4 on columns first..last */
        int64_t checkpoint = first, segments = 0;
        while (checkpoint <= last && segments < y) {
            int64_t longest = 0;
            for (int64_t i = 1; i <= 2 * E + 1; ++i) {
                int64_t len = 0;
                for (int64_t j = checkpoint; j <= last; ++j) {
                    if (sso_cell(Q, R, m, E, i, j) != 0)
                        break;
                    ++len;
                }
                if (len > longest)
                    longest = len;
            }
            if (checkpoint + longest > last)
                break; /* reached the sub-maze's last column */
            segments += 1;
            checkpoint = checkpoint + longest + 1;
        }
        count += segments;
    }
    if (count > E + 1)
        count = E + 1;
    if (accept)
        *accept = (uint8_t)(count <= E);
    if (obstacles)
        *obstacles = count;
    return SSO_OK;
}

int sso_min_obstacles(const uint8_t *Q, const uint8_t *R, int64_t m,
                      int64_t E, int64_t *out)
{
    if (m < 0 || E < 0)
        return SSO_ERR_INVALID_ARG;
    if (!valid_sequence(Q, m) || !valid_sequence(R, m))
        return SSO_ERR_INVALID_BASE;
    /* g[c] = fewest obstacles on any chain of escape segments from
     * checkpoint c (1 <= c <= m+1) to the destination.  From checkpoint c an
     * escape segment lies in one row: zeros in columns c..e-1 of that row and
     * one obstacle (any entry) at column e, after which the next checkpoint
     * is e+1; or zeros from c to column m, which ends the net with no
     * obstacle. */
    int64_t *g = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 2));
    if (!g)
        return SSO_ERR_INVALID_ARG;
    g[m + 1] = 0;
    for (int64_t c = m; c >= 1; --c) {
        int64_t best = INT64_MAX;
        for (int64_t i = 1; i <= 2 * E + 1; ++i) {
            /* e runs over every column this row's segment can end on. */
            for (int64_t e = c; e <= m; ++e) {
                int64_t cost = 1 + g[e + 1];
                if (cost < best)
                    best = cost;
                if (sso_cell(Q, R, m, E, i, e) != 0)
                    break; /* a segment holds at most one obstacle */
                if (e == m)
                    best = 0; /* zeros all the way to the row end */
            }
        }
        g[c] = best;
    }
    *out = g[1];
    free(g);
    return SSO_OK;
}

int64_t sso_edit_distance(const uint8_t *a, int64_t la, const uint8_t *b,
                          int64_t lb)
{
    int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(lb + 1));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(lb + 1));
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return -1;
    }
    for (int64_t y = 0; y <= lb; ++y)
        prev[y] = y;
    for (int64_t x = 1; x <= la; ++x) {
        cur[0] = x;
        for (int64_t y = 1; y <= lb; ++y) {
            int64_t sub = prev[y - 1] + (same_symbol(a[x - 1], b[y - 1]) ? 0 : 1);
            int64_t del = prev[y] + 1;
            int64_t ins = cur[y - 1] + 1;
            int64_t v = sub < del ? sub : del;
            cur[y] = v < ins ? v : ins;
        }
        int64_t *t = prev;
        prev = cur;
        cur = t;
    }
    int64_t d = prev[lb];
    free(prev);
    free(cur);
    return d;
}

int sso_pack_reference(const uint8_t *seq, int64_t m, uint32_t *out)
{
    int64_t words = (m + 15) / 16;
    for (int64_t w = 0; w < words; ++w)
        out[w] = 0;
    for (int64_t j = 0; j < m; ++j) {
        uint32_t code;
        switch (base_of(seq[j])) {
        case 'A': code = 0; break;
        case 'C': code = 1; break;
        case 'G': code = 2; break;
        case 'T': code = 3; break;
        default: return SSO_ERR_INVALID_BASE;
        }
        uint32_t lo = code & 1u, hi = (code >> 1) & 1u;
        out[j / 16] |= (lo << (j % 16)) | (hi << (16 + j % 16));
    }
    return SSO_OK;
}

int sso_pack_sliced(const uint8_t *seq, int64_t n, int64_t m, uint32_t *out)
{
    const int64_t G = (n + 31) / 32;
    const int64_t words = 8 * ((m + 3) / 4) * G;
    for (int64_t w = 0; w < words; ++w)
        out[w] = 0;
    for (int64_t p = 0; p < n; ++p) {
        const int64_t g = p / 32;
        const uint32_t bit = 1u << (p % 32);
        for (int64_t j = 0; j < m; ++j) {
            uint32_t code;
            switch (base_of(seq[p * m + j])) {
            case 'A': code = 0; break;
            case 'C': code = 1; break;
            case 'G': code = 2; break;
            case 'T': code = 3; break;
            default: return SSO_ERR_INVALID_BASE;
            }
            for (int b = 0; b < 2; ++b)
                if ((code >> b) & 1u)
                    out[((j / 4 * G + g) * 2 + b) * 4 + j % 4] |= bit;
        }
    }
    return SSO_OK;
}

int sso_default_threads(void)
{
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* ---- batch over host threads ------------------------------------------ */

typedef struct batch_job {
    const uint8_t *reads, *refs;
    const int64_t *offsets;
    const int32_t *lengths, *Es;
    int64_t begin, end;
    uint8_t *accept;
    int32_t *obstacles;
    sso_stats stats;
    int status;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *jb = (batch_job *)arg;
    jb->status = SSO_OK;
    for (int64_t p = jb->begin; p < jb->end; ++p) {
        int64_t m = jb->offsets ? jb->lengths[p] : jb->lengths[0];
        int64_t off = jb->offsets ? jb->offsets[p] : p * m;
        uint8_t acc = 0;
        int64_t obs = 0;
        sso_stats st;
        int rc = sso_filter(jb->reads + off, jb->refs + off, m, jb->Es[p], 1,
                            &acc, &obs, &st);
        if (rc != SSO_OK) {
            if (jb->status == SSO_OK)
                jb->status = rc;
            jb->accept[p] = 0;
            jb->obstacles[p] = -1;
            continue;
        }
        jb->accept[p] = acc;
        jb->obstacles[p] = (int32_t)obs;
        jb->stats.cells += st.cells;
        jb->stats.words += st.words;
        jb->stats.iterations += st.iterations;
        jb->stats.columns += st.columns;
    }
    return NULL;
}

int sso_filter_batch(const uint8_t *reads, const uint8_t *refs,
                     const int64_t *offsets, const int32_t *lengths,
                     const int32_t *Es, int64_t n, int threads,
                     uint8_t *accept, int32_t *obstacles,
                     sso_stats *stats_sum)
{
    if (n < 0 || (n > 0 && (!reads || !refs || !lengths || !Es)))
        return SSO_ERR_INVALID_ARG;
    for (int64_t p = 0; p < n; ++p)
        if (Es[p] < 0 || (offsets ? lengths[p] : lengths[0]) < 0)
            return SSO_ERR_INVALID_ARG;
    if (threads <= 0)
        threads = sso_default_threads();
    if (threads > n)
        threads = n > 0 ? (int)n : 1;
    batch_job *jobs = (batch_job *)calloc((size_t)threads, sizeof(batch_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tids) {
        free(jobs);
        free(tids);
        return SSO_ERR_INVALID_ARG;
    }
    for (int t = 0; t < threads; ++t) {
        batch_job *jb = &jobs[t];
        jb->reads = reads;
        jb->refs = refs;
        jb->offsets = offsets;
        jb->lengths = lengths;
        jb->Es = Es;
        jb->begin = n * t / threads;
        jb->end = n * (t + 1) / threads;
        jb->accept = accept;
        jb->obstacles = obstacles;
        pthread_create(&tids[t], NULL, batch_worker, jb);
    }
    int status = SSO_OK;
    sso_stats sum = {0, 0, 0, 0};
    for (int t = 0; t < threads; ++t) {
        pthread_join(tids[t], NULL);
        if (jobs[t].status != SSO_OK && status == SSO_OK)
            status = jobs[t].status;
        sum.cells += jobs[t].stats.cells;
        sum.words += jobs[t].stats.words;
        sum.iterations += jobs[t].stats.iterations;
        sum.columns += jobs[t].stats.columns;
    }
    if (stats_sum)
        *stats_sum = sum;
    free(jobs);
    free(tids);
    return status;
}

/* ---- unequal lengths (Section 2.4, the leading/trailing correction) ------ */

/* Eq. 1 for a query Q[1..mQ] and a reference R[1..mR]; column j = 1..mR
 * compares R[j] with Q[q], q as in sso_cell.  A cell whose q falls outside
 * 1..mQ is case 4.  With equal lengths such a cell is an obstacle (this is
 * sso_cell).  With different lengths the obstacles case 4 puts before the
 * query's first base (q < 1) or after its last (q > mQ) are the leading and
 * trailing obstacles the paper deducts from the count: here they are not
 * obstacles at all, so the net passes them free. */
int sso_cell2(const uint8_t *Q, int64_t mQ, const uint8_t *R, int64_t mR,
              int64_t E, int64_t i, int64_t j)
{
    int64_t q;
    if (i == E + 1)
        q = j;
    else if (i >= 1 && i <= E)
        q = j - i;
    else
        q = j + i - E - 1;
    if (q < 1 || q > mQ)
        return mQ == mR ? 1 : 0;
    return base_of(Q[q - 1]) == base_of(R[j - 1]) ? 0 : 1;
}

/* Section 2.4 steps (1)-(5) on the maze of sso_cell2 (mR columns).  With
 * mQ == mR this is sso_filter. */
int sso_filter2(const uint8_t *Q, int64_t mQ, const uint8_t *R, int64_t mR,
                int64_t E, int stop_above_E, uint8_t *accept,
                int64_t *obstacles)
{
    if (mQ < 0 || mR < 0 || E < 0)
        return SSO_ERR_INVALID_ARG;
    if (!valid_sequence(Q, mQ) || !valid_sequence(R, mR))
        return SSO_ERR_INVALID_BASE;
    int64_t checkpoint = 1, count = 0;
    while (checkpoint <= mR) {
        /* step (2): the longest run of zeros from the checkpoint */
        int64_t longest = 0;
        for (int64_t i = 1; i <= 2 * E + 1; ++i) {
            int64_t len = 0;
            for (int64_t j = checkpoint; j <= mR; ++j) {
                if (sso_cell2(Q, mQ, R, mR, E, i, j) != 0)
                    break;
                ++len;
            }
            if (len > longest)
                longest = len;
        }
        if (checkpoint + longest > mR)
            break; /* reached the destination */
        count += 1;                            /* the obstacle after it */
        checkpoint = checkpoint + longest + 1; /* step (3) */
        if (stop_above_E && count > E)         /* step (4) */
            break;
    }
    if (accept)
        *accept = (uint8_t)(count <= E); /* step (5) */
    if (obstacles)
        *obstacles = count;
    return SSO_OK;
}

typedef struct batch2_job {
    const uint8_t *reads, *refs;
    const int64_t *read_off, *ref_off;
    const int32_t *read_len, *ref_len, *Es;
    int64_t begin, end;
    uint8_t *accept;
    int32_t *obstacles;
    int status;
} batch2_job;

static void *batch2_worker(void *arg)
{
    batch2_job *jb = (batch2_job *)arg;
    jb->status = SSO_OK;
    for (int64_t p = jb->begin; p < jb->end; ++p) {
        uint8_t acc = 0;
        int64_t obs = 0;
        int rc = sso_filter2(jb->reads + jb->read_off[p], jb->read_len[p],
                             jb->refs + jb->ref_off[p], jb->ref_len[p],
                             jb->Es[p], 1, &acc, &obs);
        if (rc != SSO_OK) {
            if (jb->status == SSO_OK)
                jb->status = rc;
            jb->accept[p] = 0;
            jb->obstacles[p] = -1;
            continue;
        }
        jb->accept[p] = acc;
        jb->obstacles[p] = (int32_t)obs;
    }
    return NULL;
}

int sso_filter2_batch(const uint8_t *reads, const int64_t *read_off,
                      const int32_t *read_len, const uint8_t *refs,
                      const int64_t *ref_off, const int32_t *ref_len,
                      const int32_t *Es, int64_t n, int threads,
                      uint8_t *accept, int32_t *obstacles)
{
    if (n < 0 || (n > 0 && (!reads || !refs || !read_off || !read_len ||
                            !ref_off || !ref_len || !Es)))
        return SSO_ERR_INVALID_ARG;
    for (int64_t p = 0; p < n; ++p)
        if (Es[p] < 0 || read_len[p] < 0 || ref_len[p] < 0)
            return SSO_ERR_INVALID_ARG;
    if (threads <= 0)
        threads = sso_default_threads();
    if (threads > n)
        threads = n > 0 ? (int)n : 1;
    batch2_job *jobs =
        (batch2_job *)calloc((size_t)threads, sizeof(batch2_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tids) {
        free(jobs);
        free(tids);
        return SSO_ERR_INVALID_ARG;
    }
    for (int t = 0; t < threads; ++t) {
        batch2_job *jb = &jobs[t];
        jb->reads = reads;
        jb->refs = refs;
        jb->read_off = read_off;
        jb->ref_off = ref_off;
        jb->read_len = read_len;
        jb->ref_len = ref_len;
        jb->Es = Es;
        jb->begin = n * t / threads;
        jb->end = n * (t + 1) / threads;
        jb->accept = accept;
        jb->obstacles = obstacles;
        pthread_create(&tids[t], NULL, batch2_worker, jb);
    }
    int status = SSO_OK;
    for (int t = 0; t < threads; ++t) {
        pthread_join(tids[t], NULL);
        if (jobs[t].status != SSO_OK && status == SSO_OK)
            status = jobs[t].status;
    }
    free(jobs);
    free(tids);
    return status;
}

/* ---- exhaustive lower-bound check -------------------------------------- */

typedef struct exh_job {
    int m, Emax;
    int64_t begin, end; /* range of Q indices in base-4 enumeration */
    int64_t violations, pairs;
} exh_job;

static void decode4(int64_t code, int m, uint8_t *out)
{
    static const uint8_t alpha[4] = {'A', 'C', 'G', 'T'};
    for (int k = 0; k < m; ++k) {
        out[k] = alpha[code & 3];
        code >>= 2;
    }
}

static void *exh_worker(void *arg)
{
    exh_job *jb = (exh_job *)arg;
    int m = jb->m;
    int64_t total = (int64_t)1 << (2 * m);
    uint8_t Q[32], R[32];
    for (int64_t qi = jb->begin; qi < jb->end; ++qi) {
        decode4(qi, m, Q);
        for (int64_t ri = 0; ri < total; ++ri) {
            decode4(ri, m, R);
            int64_t ed = sso_edit_distance(Q, m, R, m);
            for (int E = 0; E <= jb->Emax; ++E) {
                uint8_t acc;
                int64_t obs;
                sso_filter(Q, R, m, E, 1, &acc, &obs, NULL);
                if (obs > ed || (ed <= E && !acc))
                    jb->violations += 1;
            }
            jb->pairs += 1;
        }
    }
    return NULL;
}

int64_t sso_exhaustive_lower_bound(int m, int Emax, int threads,
                                   int64_t *pairs)
{
    if (m < 0 || m > 8 || Emax < 0)
        return -1;
    if (threads <= 0)
        threads = sso_default_threads();
    int64_t total = (int64_t)1 << (2 * m);
    if (threads > total)
        threads = (int)total;
    exh_job *jobs = (exh_job *)calloc((size_t)threads, sizeof(exh_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    for (int t = 0; t < threads; ++t) {
        jobs[t].m = m;
        jobs[t].Emax = Emax;
        jobs[t].begin = total * t / threads;
        jobs[t].end = total * (t + 1) / threads;
        pthread_create(&tids[t], NULL, exh_worker, &jobs[t]);
    }
    int64_t v = 0, p = 0;
    for (int t = 0; t < threads; ++t) {
        pthread_join(tids[t], NULL);
        v += jobs[t].violations;
        p += jobs[t].pairs;
    }
    free(jobs);
    free(tids);
    if (pairs)
        *pairs = p;
    return v;
}
