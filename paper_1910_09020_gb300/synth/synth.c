/*
 * synth.c -- seeded synthetic read/reference pairs.
 *
 * This module only draws random sequences and random edits.  It holds none
 * of the filter's arithmetic, so both the CUDA path and the CPU oracle may be
 * fed from it.  Every pair is generated from its own counter-based stream
 * (splitmix64 keyed by seed and pair index), so any subset of pairs, on any
 * number of threads, in any order, comes out identical.
 *
 * Shapes follow the paper's workloads (Section 3.1): uniform i.i.d. ACGT
 * reads; the reference segment is the read with random substitutions,
 * insertions and deletions, then cut or padded with random bases back to the
 * read's length (equal-length pairs, the paper's Section 2.3 assumption).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

enum {
    SYN_EDITS_UNIFORM_K = 0, /* k ~ U{kmin..kmax} edits, types by psub/pins/pdel */
    SYN_EDITS_POISSON = 1,   /* k ~ Poisson(lambda); odd pairs independent random */
    SYN_EDITS_RATE = 2       /* each base edited w.p. r, r ~ U[0, rmax] per pair */
};

typedef struct syn_params {
    int32_t mode;
    int32_t kmin, kmax;
    double lambda;
    double rmax;
    double psub, pins, pdel;
} syn_params;

typedef struct rng {
    uint64_t s;
} rng;

static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static rng pair_stream(uint64_t seed, int64_t pair, uint64_t salt)
{
    rng r;
    uint64_t k = seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(pair + 1)) ^ salt;
    r.s = splitmix64(&k);
    return r;
}

static uint64_t next_u64(rng *r) { return splitmix64(&r->s); }

static double next_unit(rng *r) /* [0, 1) */
{
    return (double)(next_u64(r) >> 11) * (1.0 / 9007199254740992.0);
}

static uint32_t next_below(rng *r, uint32_t n) /* [0, n) */
{
    return (uint32_t)(((next_u64(r) >> 32) * (uint64_t)n) >> 32);
}

static const uint8_t ALPHA[4] = {'A', 'C', 'G', 'T'};

static uint8_t random_base(rng *r) { return ALPHA[next_below(r, 4)]; }

static uint8_t other_base(rng *r, uint8_t b)
{
    uint8_t c;
    do {
        c = random_base(r);
    } while (c == b);
    return c;
}

static int poisson(rng *r, double lambda)
{
    double L = exp(-lambda), p = 1.0;
    int k = 0;
    do {
        ++k;
        p *= next_unit(r);
    } while (p > L && k < 100000);
    return k - 1;
}

/* One edit of a chosen type at a uniform position of buf[0..*len). */
static void apply_edit(rng *r, uint8_t *buf, int64_t *len, int64_t cap,
                       int type)
{
    if (type == 0) { /* substitution */
        if (*len == 0)
            return;
        int64_t pos = next_below(r, (uint32_t)*len);
        buf[pos] = other_base(r, buf[pos]);
    } else if (type == 1) { /* insertion */
        if (*len >= cap)
            return;
        int64_t pos = next_below(r, (uint32_t)(*len + 1));
        memmove(buf + pos + 1, buf + pos, (size_t)(*len - pos));
        buf[pos] = random_base(r);
        *len += 1;
    } else { /* deletion */
        if (*len == 0)
            return;
        int64_t pos = next_below(r, (uint32_t)*len);
        memmove(buf + pos, buf + pos + 1, (size_t)(*len - pos - 1));
        *len -= 1;
    }
}

static int draw_type(rng *r, const syn_params *p)
{
    double u = next_unit(r) * (p->psub + p->pins + p->pdel);
    if (u < p->psub)
        return 0;
    if (u < p->psub + p->pins)
        return 1;
    return 2;
}

/* Generate pair `pair` of length m into read/ref (m bytes each).  work must
 * hold 2m + 16 bytes. */
static void gen_pair(uint64_t seed, int64_t pair, int64_t m,
                     const syn_params *p, uint8_t *read, uint8_t *ref,
                     uint8_t *work)
{
    rng r = pair_stream(seed, pair, 0x5EEDull);
    for (int64_t j = 0; j < m; ++j)
        read[j] = random_base(&r);
    int64_t cap = 2 * m + 8;
    int64_t len = 0;

    if (p->mode == SYN_EDITS_POISSON && (pair & 1)) {
        /* independent random reference */
        for (int64_t j = 0; j < m; ++j)
            ref[j] = random_base(&r);
        return;
    }
    if (p->mode == SYN_EDITS_RATE) {
        double rate = next_unit(&r) * p->rmax;
        for (int64_t j = 0; j < m && len < cap; ++j) {
            if (next_unit(&r) < rate) {
                int t = draw_type(&r, p);
                if (t == 0) {
                    work[len++] = other_base(&r, read[j]);
                } else if (t == 1) {
                    work[len++] = random_base(&r);
                    if (len < cap)
                        work[len++] = read[j];
                } /* deletion: skip read[j] */
            } else {
                work[len++] = read[j];
            }
        }
    } else {
        memcpy(work, read, (size_t)m);
        len = m;
        int k;
        if (p->mode == SYN_EDITS_POISSON)
            k = poisson(&r, p->lambda);
        else
            k = p->kmin + (int)next_below(&r, (uint32_t)(p->kmax - p->kmin + 1));
        for (int e = 0; e < k; ++e)
            apply_edit(&r, work, &len, cap, draw_type(&r, p));
    }
    /* cut or pad with random bases back to m */
    for (int64_t j = 0; j < m; ++j)
        ref[j] = j < len ? work[j] : random_base(&r);
}

/* ---- public entry points ------------------------------------------------ */

typedef struct job {
    uint64_t seed;
    int64_t first, begin, end;
    const int64_t *offsets;
    const int32_t *lengths;
    int32_t m;
    const syn_params *p;
    uint8_t *reads, *refs;
} job;

static void *worker(void *arg)
{
    job *jb = (job *)arg;
    int64_t maxm = jb->m;
    if (jb->offsets)
        for (int64_t i = jb->begin; i < jb->end; ++i)
            if (jb->lengths[i] > maxm)
                maxm = jb->lengths[i];
    uint8_t *work = (uint8_t *)malloc((size_t)(2 * maxm + 16));
    for (int64_t i = jb->begin; i < jb->end; ++i) {
        int64_t m = jb->offsets ? jb->lengths[i] : jb->m;
        int64_t off = jb->offsets ? jb->offsets[i] : i * (int64_t)jb->m;
        gen_pair(jb->seed, jb->first + i, m, jb->p, jb->reads + off,
                 jb->refs + off, work);
    }
    free(work);
    return NULL;
}

static int nthreads(int threads, int64_t n)
{
    if (threads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        threads = c > 0 ? (int)c : 1;
    }
    if (threads > n)
        threads = n > 0 ? (int)n : 1;
    return threads;
}

/* Pairs first..first+n-1.  offsets == NULL: fixed length m, pair i at byte
 * i*m.  Otherwise pair i has length lengths[i] at byte offsets[i]. */
int synth_pairs(uint64_t seed, int64_t first, int64_t n, int32_t m,
                const int64_t *offsets, const int32_t *lengths,
                const syn_params *p, uint8_t *reads, uint8_t *refs,
                int threads)
{
    if (n <= 0)
        return 0;
    int T = nthreads(threads, n);
    job *jobs = (job *)calloc((size_t)T, sizeof(job));
    pthread_t *tid = (pthread_t *)calloc((size_t)T, sizeof(pthread_t));
    for (int t = 0; t < T; ++t) {
        jobs[t] = (job){seed,     first,   n * t / T, n * (t + 1) / T,
                        offsets,  lengths, m,         p,
                        reads,    refs};
        pthread_create(&tid[t], NULL, worker, &jobs[t]);
    }
    for (int t = 0; t < T; ++t)
        pthread_join(tid[t], NULL);
    free(jobs);
    free(tid);
    return 0;
}

/* Log-uniform integers floor(exp(U[ln lo, ln hi])) clamped to [lo, hi], one
 * per pair (pair-indexed streams, like the sequences). */
int synth_log_uniform(uint64_t seed, int64_t first, int64_t n, double lo,
                      double hi, uint64_t salt, int32_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        rng r = pair_stream(seed, first + i, salt);
        double u = next_unit(&r);
        double v = floor(exp(log(lo) + u * (log(hi) - log(lo))));
        if (v < lo)
            v = lo;
        if (v > hi)
            v = hi;
        out[i] = (int32_t)v;
    }
    return 0;
}

/* Exponential inter-arrival gaps (mean 1/rate) for Poisson arrivals. */
int synth_poisson_arrivals(uint64_t seed, int64_t n, double rate, double *out)
{
    rng r = pair_stream(seed, 0, 0xA77Eull);
    double t = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double u = next_unit(&r);
        t += -log(1.0 - u) / rate;
        out[i] = t;
    }
    return 0;
}
