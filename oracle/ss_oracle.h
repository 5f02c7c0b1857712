/*
 * ss_oracle.h -- plain, slow CPU SneakySnake used as the parity oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path includes, links or
 * calls this code: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * library; the two meet only through the seeded input generator.
 *
 * Conventions follow the paper (Alser et al., SneakySnake, Section 2.3-2.4):
 *   R[1..m]  reference sequence, Q[1..m] query (read) sequence, both ASCII.
 *   E        edit distance threshold.
 *   Z[i, j]  chip maze entry, 1 <= i <= 2E+1 (HRTs), 1 <= j <= m (VRTs); 0 =
 *            available path, 1 = obstacle (Eq. 1).
 * Bases are A, C, G, T in either case; any other byte is invalid (the paper
 * is silent on other symbols; this oracle rejects them).
 */
#ifndef SS_ORACLE_H
#define SS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define SSO_OK 0
#define SSO_ERR_INVALID_ARG (-1)
#define SSO_ERR_INVALID_BASE (-2)

/* Work counters of one greedy run (used to state the op model of the
 * roofline).  cells: maze entries evaluated by the implicit maze of Section
 * 2.4 (from each checkpoint up to and including the first obstacle of every
 * row, or up to the row end); words: the same cells counted in 32-column
 * words per row and checkpoint (ceil(cells_in_row / 32)); iterations: number
 * of checkpoints visited (escape segments searched); columns: maze columns
 * those searches span (from each checkpoint through the column of the
 * segment's obstacle, or to the row end) -- what a walk that evaluates all
 * 2E+1 rows of one column at a time visits. */
typedef struct sso_stats {
    int64_t cells;
    int64_t words;
    int64_t iterations;
    int64_t columns;
} sso_stats;

/* Eq. 1: the chip maze entry Z[i, j] (1-based i, j).  Returns 0 or 1. */
int sso_cell(const uint8_t *Q, const uint8_t *R, int64_t m, int64_t E,
             int64_t i, int64_t j);

/* Fill Z (row-major, (2E+1) x m bytes of 0/1) with the complete chip maze of
 * Fig. 2(b).  Returns SSO_OK or an error code. */
int sso_maze(const uint8_t *Q, const uint8_t *R, int64_t m, int64_t E,
             uint8_t *Z);

/* The SneakySnake filter of Section 2.4, steps (1)-(5), on the implicit maze.
 * stop_above_E = 1 is the paper's step (4) (stop once the obstacle count
 * exceeds E); 0 keeps routing to the destination terminal (used only by the
 * optimality check of Theorem 2).  Writes accept (count <= E) and the
 * obstacle count (capped at E+1 when stop_above_E = 1).  stats may be NULL. */
int sso_filter(const uint8_t *Q, const uint8_t *R, int64_t m, int64_t E,
               int stop_above_E, uint8_t *accept, int64_t *obstacles,
               sso_stats *stats);

/* Snake-on-Chip's decomposition (Section 2.5): the maze is cut into
 * sub-mazes of t consecutive columns (the last may be narrower), each routed
 * independently by the greedy of Section 2.4 from its first column to its
 * last (a run reaching the sub-maze's last column ends it without an
 * obstacle).  Reading of the y "module instances per sub-maze": at most y
 * escape segments are routed per sub-maze, so a sub-maze contributes at most
 * y obstacles.  Sub-maze counts are summed, stopping once the sum exceeds
 * E; accept = (sum <= E), obstacles = min(sum, E+1).  The decomposition can
 * only underestimate the full greedy count (the paper says so). */
int sso_filter_submaze(const uint8_t *Q, const uint8_t *R, int64_t m,
                       int64_t E, int64_t t, int64_t y, uint8_t *accept,
                       int64_t *obstacles);

/* Unequal lengths (Section 2.4's correction for sequences of different
 * length).  The maze has mR columns (one per reference base, as Eq. 1
 * compares R[j]) and 2E+1 rows; a cell whose query index q falls outside
 * 1..mQ is case 4.  Reading of "deduct the leading and trailing obstacles
 * caused by the fourth case": when mQ != mR those cells (q < 1: before the
 * query's first base; q > mQ: after its last) are not obstacles, so the net
 * passes the sequences' overhanging ends free; when mQ == mR nothing changes
 * (sso_cell2 == sso_cell, sso_filter2 == sso_filter). */
int sso_cell2(const uint8_t *Q, int64_t mQ, const uint8_t *R, int64_t mR,
              int64_t E, int64_t i, int64_t j);
int sso_filter2(const uint8_t *Q, int64_t mQ, const uint8_t *R, int64_t mR,
                int64_t E, int stop_above_E, uint8_t *accept,
                int64_t *obstacles);
/* Batch of sso_filter2 over host threads: pair p is Q = reads +
 * read_off[p] (read_len[p] bases), R = refs + ref_off[p] (ref_len[p] bases),
 * threshold Es[p].  Invalid pairs get obstacles -1 and the first error is
 * returned. */
int sso_filter2_batch(const uint8_t *reads, const int64_t *read_off,
                      const int32_t *read_len, const uint8_t *refs,
                      const int64_t *ref_off, const int32_t *ref_len,
                      const int32_t *Es, int64_t n, int threads,
                      uint8_t *accept, int32_t *obstacles);

/* Minimum number of obstacles over every chain of non-overlapping escape
 * segments that links column 1 to the destination terminal (the optimum
 * Theorem 2 says the greedy reaches), by dynamic programming over
 * checkpoints.  O(m^2 (2E+1)) -- small inputs only. */
int sso_min_obstacles(const uint8_t *Q, const uint8_t *R, int64_t m,
                      int64_t E, int64_t *out);

/* Levenshtein (edit) distance between a[0..la) and b[0..lb) by the textbook
 * dynamic program (unit cost substitution, insertion, deletion). */
int64_t sso_edit_distance(const uint8_t *a, int64_t la, const uint8_t *b,
                          int64_t lb);

/* Batch filter over n pairs on `threads` host threads (0 = all cores).
 * Pair p uses Q = reads + offsets[p], R = refs + offsets[p], length
 * lengths[p] and threshold Es[p].  offsets may be NULL, meaning a fixed
 * stride of lengths[0] (then every pair has length lengths[0]).  Returns
 * SSO_OK, or the first error met (pairs with invalid bases give
 * SSO_ERR_INVALID_BASE).  stats_sum may be NULL; else it receives the sum of
 * the per-pair counters. */
int sso_filter_batch(const uint8_t *reads, const uint8_t *refs,
                     const int64_t *offsets, const int32_t *lengths,
                     const int32_t *Es, int64_t n, int threads,
                     uint8_t *accept, int32_t *obstacles,
                     sso_stats *stats_sum);

/* Exhaustive check of the lower-bound property (Theorem 2, 0 % false
 * reject): for every pair of ACGT strings of length m and every E in
 * [0, Emax], min(count, E+1) <= edit distance and (ED <= E => accept).
 * Returns the number of violations; *pairs receives the number of pairs
 * tested. */
int64_t sso_exhaustive_lower_bound(int m, int Emax, int threads,
                                   int64_t *pairs);

/* Reference packer of the library's 2-bit packed format, written from its
 * written definition (not from the library): base j of a sequence goes to
 * 32-bit word j/16; bit (j%16) of that word holds bit 0 of the base code and
 * bit 16+(j%16) holds bit 1, with codes A=0, C=1, G=2, T=3 (either case).
 * Unused bits are zero.  out has ceil(m/16) words.  Returns SSO_OK or
 * SSO_ERR_INVALID_BASE. */
int sso_pack_reference(const uint8_t *seq, int64_t m, uint32_t *out);

/* Reference packer of the library's bit-sliced format, written from its
 * written definition: n sequences of m bases (sequence p at seq + p*m) in
 * groups of 32 (sequence p is bit p%32 of group p/32, G = ceil(n/32)
 * groups); bit b (0 or 1) of the code of base j of the group's sequences
 * forms one 32-bit word, stored at index ((j/4 * G + g) * 2 + b) * 4 + j%4.
 * Codes as above; bits of sequences p >= n and words of bases j >= m are
 * zero.  out has 8 * ceil(m/4) * G words.  Returns SSO_OK or
 * SSO_ERR_INVALID_BASE. */
int sso_pack_sliced(const uint8_t *seq, int64_t n, int64_t m, uint32_t *out);

/* Number of host threads the batch routines use for threads = 0. */
int sso_default_threads(void);

#ifdef __cplusplus
}
#endif
#endif
