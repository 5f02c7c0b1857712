"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each ``pin_*`` takes an :class:`oracle.Oracle` and raises AssertionError when
the oracle disagrees with the fact it checks.  ``test_oracle_pins.py`` runs
them on the real oracle; ``test_oracle_mutants.py`` runs them on copies of the
oracle with planted mistakes and requires every mistake to be caught.

Sources of truth (none of them is the oracle itself):
* the worked example of Fig. 2 / Fig. 1 (R, Q, E = 3, 7 x 12 maze, 3
  obstacles, accept) from ``tests/golden/fig2_worked_example.txt``;
* the row count 2E+1 (E = 5010 gives 10,021 rows, Section 3.5);
* Theorem 2 (the count is the minimum over all chains of escape segments,
  and a lower bound on edit distance: no false rejects), checked by brute
  force and by an independent dynamic program;
* closed forms: identical pairs, E = 0, one substitution, one indel, the
  Hamming bound, monotonicity in E;
* textbook edit distances and a breadth-first search over edit scripts;
* for pairs of different lengths: closed forms (a reference that extends the
  query costs nothing), a banded semi-global dynamic program (no false
  reject for approximate string matching) and Theorem 2's optimality on the
  corrected maze.
"""
from __future__ import annotations

import collections
import os
import random

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "fig2_worked_example.txt")
ALPHA = "ACGT"


def load_golden(path: str = GOLDEN) -> dict:
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(None, 1)
            out[k] = v
    return out


def rand_seq(rng: random.Random, m: int) -> str:
    return "".join(rng.choice(ALPHA) for _ in range(m))


def mutate(rng: random.Random, s: str, k: int) -> str:
    """k random edits (substitution / insertion / deletion), then cut or pad
    to len(s) -- a small local stand-in for the workload generator."""
    t = list(s)
    for _ in range(k):
        op = rng.randrange(3)
        if op == 0 and t:
            p = rng.randrange(len(t))
            t[p] = rng.choice([c for c in ALPHA if c != t[p]])
        elif op == 1:
            t.insert(rng.randrange(len(t) + 1), rng.choice(ALPHA))
        elif t:
            del t[rng.randrange(len(t))]
    t = t[: len(s)]
    while len(t) < len(s):
        t.append(rng.choice(ALPHA))
    return "".join(t)


def random_pairs(seed: int, count: int, mmax: int, kmax: int):
    rng = random.Random(seed)
    for _ in range(count):
        m = rng.randint(1, mmax)
        Q = rand_seq(rng, m)
        R = mutate(rng, Q, rng.randint(0, kmax)) if rng.random() < 0.8 \
            else rand_seq(rng, m)
        yield Q, R


# ---- worked example --------------------------------------------------------

def pin_worked_example_maze(O):
    g = load_golden()
    E = int(g["E"])
    Z = O.maze(g["Q"], g["R"], E)
    assert Z.shape == (int(g["rows"]), int(g["cols"])), Z.shape
    for i in range(1, Z.shape[0] + 1):
        got = "".join(str(int(v)) for v in Z[i - 1])
        assert got == g[f"row{i}"], (i, got, g[f"row{i}"])
    col6 = "".join(str(int(v)) for v in Z[:, 5])
    assert col6 == g["col6"], col6


def pin_worked_example_decision(O):
    g = load_golden()
    res = O.filter_pair(g["Q"], g["R"], int(g["E"]))
    assert res.obstacles == int(g["obstacles"]), res
    assert res.accept == bool(int(g["accept"])), res


def pin_column6_orientation(O):
    """Fig. 2a: column 6 compares R[6] with Q[5], Q[4], Q[3] (rows 1..3, in
    that reversed order), Q[6] (row 4) and Q[7..9] (rows 5..7)."""
    g = load_golden()
    Q, R, E = g["Q"], g["R"], int(g["E"])
    order = [5, 4, 3, 6, 7, 8, 9]
    for i, q in enumerate(order, start=1):
        want = 0 if Q[q - 1] == R[5] else 1
        assert O.cell(Q, R, E, i, 6) == want, (i, q)


def pin_row_count(O):
    """2E+1 HRTs; E = 5010 gives a maze of 10,021 rows (Section 3.5)."""
    Z = O.maze("ACGT", "ACGA", 5010)
    assert Z.shape == (10021, 4)
    for E in (0, 1, 7):
        assert O.maze("ACGTA", "ACGTA", E).shape == (2 * E + 1, 5)


# ---- closed forms ----------------------------------------------------------

def pin_identical(O):
    rng = random.Random(11)
    for m in (1, 2, 31, 32, 33, 100, 257):
        Q = rand_seq(rng, m)
        for E in (0, 1, 3, 10):
            assert O.filter_pair(Q, Q, E) == (True, 0), (m, E)
    assert O.filter_pair("", "", 3) == (True, 0)


def pin_E0(O):
    """E = 0: one row, the main diagonal; accept iff Q = R; count <= 1."""
    for Q, R in random_pairs(12, 300, 120, 3):
        res = O.filter_pair(Q, R, 0)
        assert res == ((Q == R), 0 if Q == R else 1), (Q, R, res)


def pin_single_substitution(O):
    rng = random.Random(13)
    for m in (1, 2, 5, 64, 100, 150):
        Q = rand_seq(rng, m)
        for k in sorted({0, m // 2, m - 1}):
            R = Q[:k] + rng.choice([c for c in ALPHA if c != Q[k]]) + Q[k + 1:]
            for E in (1, 2, 5):
                assert O.filter_pair(Q, R, E) == (True, 1), (m, k, E)


def pin_single_indel(O):
    """Q = R with base k deleted and one base appended: the main diagonal
    matches up to column k, row i = 1 (Q[j-1]) matches from column k+2 to
    the row end, so a net of exactly one obstacle exists (none with zero
    unless Q = R).  Q = R with a base inserted at k and cut to m: the row
    i = E+2 (Q[j+1]) runs out of Q in the last column (Eq. 1 case 4), so a
    net of at most two obstacles exists -- the trailing obstacle Section 2.4
    attributes to unequal lengths."""
    rng = random.Random(14)
    for m in (3, 40, 100, 200):
        R = rand_seq(rng, m)
        for k in (1, m // 2, m - 2):
            Qd = R[:k] + R[k + 1:] + rng.choice(ALPHA)
            Qi = (R[:k] + rng.choice(ALPHA) + R[k:])[:m]
            for E in (1, 3):
                if Qd != R:
                    assert O.filter_pair(Qd, R, E) == (True, 1), (m, k, E)
                if Qi != R:
                    unc = O.filter_pair(Qi, R, E, stop_above_E=False)
                    assert 1 <= unc.obstacles <= 2, (m, k, E, unc)


def pin_hamming_bound(O):
    """The main-diagonal net has one obstacle per mismatch, so the optimum
    never exceeds the Hamming distance."""
    for Q, R in random_pairs(15, 300, 200, 12):
        ham = sum(a != b for a, b in zip(Q, R))
        for E in (0, 2, 6):
            unc = O.filter_pair(Q, R, E, stop_above_E=False).obstacles
            assert unc <= ham, (Q, R, E, unc, ham)


def pin_monotone_in_E(O):
    """More rows can only lengthen the longest run: the uncapped count does
    not grow with E."""
    for Q, R in random_pairs(16, 150, 150, 10):
        prev = None
        for E in range(0, 9):
            unc = O.filter_pair(Q, R, E, stop_above_E=False).obstacles
            if prev is not None:
                assert unc <= prev, (Q, R, E)
            prev = unc


def pin_cap(O):
    """Step (4) stops once the count exceeds E: the report is min(count,
    E+1) and accept iff count <= E."""
    for Q, R in random_pairs(17, 300, 150, 12):
        for E in (0, 1, 3, 8):
            unc = O.filter_pair(Q, R, E, stop_above_E=False).obstacles
            res = O.filter_pair(Q, R, E)
            assert res.obstacles == min(unc, E + 1), (Q, R, E)
            assert res.accept == (unc <= E), (Q, R, E)


def pin_cap_counterexample(O):
    """Q = ACA, R = CAC, E = 0: the uncapped count (3) exceeds the edit
    distance (2); the capped count (1) does not."""
    assert O.edit_distance("ACA", "CAC") == 2
    assert O.filter_pair("ACA", "CAC", 0, stop_above_E=False).obstacles == 3
    assert O.filter_pair("ACA", "CAC", 0) == (False, 1)


def pin_E_at_least_m(O):
    """Rows with |shift| >= m are all obstacles: for E >= m the count equals
    the count at E = m-1, and the pair is accepted (count <= m <= E)."""
    rng = random.Random(18)
    for m in (1, 2, 3, 7, 20):
        for _ in range(10):
            Q, R = rand_seq(rng, m), rand_seq(rng, m)
            base = O.filter_pair(Q, R, m - 1, stop_above_E=False).obstacles
            for E in (m, m + 1, 3 * m):
                assert O.filter_pair(Q, R, E, stop_above_E=False).obstacles \
                    == base
                assert O.filter_pair(Q, R, E).accept


# ---- Theorem 2 ---------------------------------------------------------------

def pin_optimality(O):
    """Theorem 2: the greedy count equals the minimum over every chain of
    non-overlapping escape segments (independent dynamic program)."""
    for Q, R in random_pairs(19, 120, 90, 12):
        for E in (0, 1, 2, 4, 7):
            unc = O.filter_pair(Q, R, E, stop_above_E=False).obstacles
            assert unc == O.min_obstacles(Q, R, E), (Q, R, E)


def pin_lower_bound_random(O):
    """Theorem 2 / 0 % false reject: min(count, E+1) <= edit distance, and
    every pair within E edits is accepted."""
    for Q, R in random_pairs(20, 250, 300, 15):
        ed = O.edit_distance(Q, R)
        for E in (0, 1, 3, 5, 10, 15):
            res = O.filter_pair(Q, R, E)
            assert res.obstacles <= ed, (Q, R, E, res, ed)
            if ed <= E:
                assert res.accept, (Q, R, E, ed)


def pin_lower_bound_exhaustive(O, mmax: int = 5, Emax: int = 3):
    for m in range(1, mmax + 1):
        v, n = O.exhaustive_lower_bound(m, Emax)
        assert n == 4 ** (2 * m), (m, n)
        assert v == 0, (m, v)


# ---- edit distance -------------------------------------------------------------

def pin_edit_distance_textbook(O):
    assert O.edit_distance("kitten", "sitting") == 3
    assert O.edit_distance("flaw", "lawn") == 2
    assert O.edit_distance("intention", "execution") == 5
    assert O.edit_distance("", "ACGT") == 4
    assert O.edit_distance("ACGT", "") == 4
    assert O.edit_distance("ACGT", "ACGT") == 0


def _bfs_distance(a: str, b: str) -> int:
    """Fewest single-base substitutions, insertions and deletions that turn a
    into b, by breadth-first search over strings (no dynamic program)."""
    cap = max(len(a), len(b))
    seen = {a: 0}
    dq = collections.deque([a])
    while dq:
        s = dq.popleft()
        d = seen[s]
        if s == b:
            return d
        nxt = []
        for p in range(len(s)):
            nxt.append(s[:p] + s[p + 1:])
            for c in ALPHA:
                if c != s[p]:
                    nxt.append(s[:p] + c + s[p + 1:])
        if len(s) < cap:
            for p in range(len(s) + 1):
                for c in ALPHA:
                    nxt.append(s[:p] + c + s[p:])
        for t in nxt:
            if t not in seen:
                seen[t] = d + 1
                dq.append(t)
    raise AssertionError("unreachable")


def pin_edit_distance_bfs(O):
    rng = random.Random(21)
    for _ in range(150):
        a = rand_seq(rng, rng.randint(0, 4))
        b = rand_seq(rng, rng.randint(0, 4))
        assert O.edit_distance(a, b) == _bfs_distance(a, b), (a, b)


# ---- input handling ---------------------------------------------------------

def pin_case_and_invalid(O):
    g = load_golden()
    lower = O.filter_pair(g["Q"].lower(), g["R"], int(g["E"]))
    assert lower == (True, 3)
    try:
        O.filter_pair("ACGN", "ACGT", 1)
    except ValueError:
        pass
    else:
        raise AssertionError("non-ACGT base accepted")


def pin_pack_reference(O):
    """The library's 2-bit format: base j -> word j/16, bit j%16 = code bit
    0, bit 16 + j%16 = code bit 1; A=0, C=1, G=2, T=3 (values by hand)."""
    assert list(O.pack_reference("ACGT")) == [0x000C000A]
    assert list(O.pack_reference("T" * 16)) == [0xFFFFFFFF]
    assert list(O.pack_reference("A" * 16 + "G")) == [0, 0x00010000]
    assert list(O.pack_reference("acgt")) == [0x000C000A]
    assert list(O.pack_reference("C" * 17)) == [0x0000FFFF, 0x00000001]


def pin_pack_sliced(O):
    """The library's bit-sliced format: sequence p is bit p%32 of group
    p/32; code bit b of base j of group g is word ((j/4*G + g)*2 + b)*4 +
    j%4.  Values by hand, then every bit against the 2-bit packer."""
    two = np.frombuffer(b"ACGTATTTTC", np.uint8).reshape(2, 5)
    # base j: (lo, hi) of seq 0 in bit 0, of seq 1 in bit 1
    #   j=0 A,T  j=1 C,T  j=2 G,T  j=3 T,T  j=4 A,C
    assert list(O.pack_sliced(two)) == [2, 3, 2, 3, 2, 2, 3, 3,
                                        2, 0, 0, 0, 0, 0, 0, 0]
    g33 = np.full((33, 1), ord("G"), np.uint8)  # two groups, G = 2
    w = O.pack_sliced(g33)
    assert len(w) == 16
    assert (w[0], w[4], w[8], w[12]) == (0, 0xFFFFFFFF, 0, 1)
    assert not w[[1, 2, 3, 5, 6, 7, 9, 10, 11, 13, 14, 15]].any()
    rng = random.Random(31)
    n, m = 70, 23
    seqs = [rand_seq(rng, m) for _ in range(n)]
    arr = np.frombuffer("".join(seqs).encode(), np.uint8).reshape(n, m)
    w = O.pack_sliced(arr)
    G = (n + 31) // 32
    assert len(w) == 8 * ((m + 3) // 4) * G
    for p in range(n):
        packed = O.pack_reference(seqs[p])
        for j in range(m):
            for b in range(2):
                want = (int(packed[j // 16]) >> (16 * b + j % 16)) & 1
                got = (int(w[((j // 4 * G + p // 32) * 2 + b) * 4 + j % 4])
                       >> (p % 32)) & 1
                assert got == want, (p, j, b)
    # nothing else set: pad sequences of the last group, bases past m
    total = sum(bin(int(x)).count("1") for x in w)
    assert total == sum(bin(int(x)).count("1")
                        for s in seqs for x in O.pack_reference(s))


def pin_batch_matches_single(O):
    rng = random.Random(22)
    n, m = 64, 70
    Qs = [rand_seq(rng, m) for _ in range(n)]
    Rs = [mutate(rng, q, rng.randint(0, 6)) for q in Qs]
    reads = np.frombuffer("".join(Qs).encode(), np.uint8).reshape(n, m)
    refs = np.frombuffer("".join(Rs).encode(), np.uint8).reshape(n, m)
    acc, obs = O.filter_batch(reads, refs, m, 3, threads=4)
    for p in range(n):
        r = O.filter_pair(Qs[p], Rs[p], 3)
        assert (bool(acc[p]), int(obs[p])) == r, p
    lens = np.array([rng.randint(0, 90) for _ in range(n)], np.int32)
    Qv = [rand_seq(rng, int(L)) for L in lens]
    Rv = [mutate(rng, q, 3) for q in Qv]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    Es = np.array([rng.randint(0, 6) for _ in range(n)], np.int32)
    acc, obs = O.filter_batch(np.frombuffer("".join(Qv).encode(), np.uint8),
                              np.frombuffer("".join(Rv).encode(), np.uint8),
                              lens, Es, offsets=off, threads=3)
    for p in range(n):
        r = O.filter_pair(Qv[p], Rv[p], int(Es[p]))
        assert (bool(acc[p]), int(obs[p])) == r, p


# ---- Snake-on-Chip decomposition (Section 2.5) -------------------------------

def pin_submaze_worked_example(O):
    g = load_golden()
    Q, R, E = g["Q"], g["R"], int(g["E"])
    for t, y in ((4, 3), (4, 1), (3, 3), (3, 1)):
        got = O.filter_submaze(Q, R, E, t, y).obstacles
        assert got == int(g[f"submaze_t{t}_y{y}"]), (t, y, got)


def pin_submaze_reduces_to_full(O):
    """One sub-maze spanning the whole maze with no segment cap is the
    greedy of Section 2.4."""
    for Q, R in random_pairs(23, 150, 120, 12):
        m = len(Q)
        for E in (0, 2, 5):
            assert O.filter_submaze(Q, R, E, m, m + 1) == \
                O.filter_pair(Q, R, E), (Q, R, E)


def pin_submaze_underestimates(O):
    """Cutting the maze can only lose obstacles (Section 2.5): the count is
    at most the full greedy's, so no pair the full filter accepts is
    rejected; a larger segment cap never lowers it."""
    for Q, R in random_pairs(24, 150, 200, 15):
        for E in (1, 4, 10):
            full = O.filter_pair(Q, R, E, stop_above_E=False).obstacles
            for t in (1, 3, 8, 31):
                prev = -1
                for y in (1, 2, 3, 100):
                    sub = O.filter_submaze(Q, R, E, t, y).obstacles
                    assert sub <= min(full, E + 1), (Q, R, E, t, y)
                    assert sub >= prev
                    prev = sub


# ---- pairs of different lengths (Section 2.4's correction) ---------------------

def _sg_band(Q: str, R: str, E: int) -> int:
    """Edit distance of Q to a stretch of R that starts within R's first E+1
    bases, every aligned position within E diagonals of the main one (the
    rows of Eq. 1); the reference bases before and after the stretch are
    free.  A plain dynamic program, independent of the oracle."""
    mq, mr = len(Q), len(R)
    inf = 10 ** 9
    D = [[inf] * (mr + 1) for _ in range(mq + 1)]
    for j in range(min(E, mr) + 1):
        D[0][j] = 0
    for i in range(1, mq + 1):
        for j in range(mr + 1):
            if abs(i - j) > E:
                continue
            best = inf
            if j and abs(i - j) <= E and D[i - 1][j - 1] < inf:
                best = min(best, D[i - 1][j - 1] + (Q[i - 1] != R[j - 1]))
            if abs(i - 1 - j) <= E and D[i - 1][j] < inf:
                best = min(best, D[i - 1][j] + 1)
            if j and abs(i - j + 1) <= E and D[i][j - 1] < inf:
                best = min(best, D[i][j - 1] + 1)
            D[i][j] = best
    ends = [D[mq][j] for j in range(mr + 1) if abs(mq - j) <= E]
    return min(ends) if ends else inf


def _unequal_pairs(seed: int, n: int, mmax: int):
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        mq = rng.randint(1, mmax)
        mr = mq + rng.choice([-3, -2, -1, 1, 2, 3, 5, 9])
        if mr < 1:
            mr = mq + 1
        Q = rand_seq(rng, mq)
        R = mutate(rng, Q, rng.randint(0, 3))
        R = (R + rand_seq(rng, mr))[:mr]
        out.append((Q, R))
    return out


def pin_unequal_equal_lengths_unchanged(O):
    """The correction is for sequences of different length only: with equal
    lengths the pair is filtered exactly as before."""
    for Q, R in random_pairs(31, 200, 80, 10):
        for E in (0, 1, 2, 4, 8):
            assert O.filter_unequal(Q, R, E) == O.filter_pair(Q, R, E), \
                (Q, R, E)


def pin_unequal_free_flanks(O):
    """Closed forms: the reference's bases before or after the query (within
    the 2E+1 rows on the left) cost nothing, in either direction of the
    length difference; at E = 0 the count is the Hamming distance of the
    overlapping prefix."""
    rng = random.Random(32)
    for _ in range(60):
        Q = rand_seq(rng, rng.randint(3, 60))
        X = rand_seq(rng, rng.randint(1, 6))
        Y = rand_seq(rng, rng.randint(1, 25))
        for E in (0, 1, 3, 6):
            assert O.filter_unequal(Q, Q + Y, E).obstacles == 0, (Q, Y, E)
            assert O.filter_unequal(Q + Y, Q, E).obstacles == 0, (Q, Y, E)
            if E >= len(X):
                assert O.filter_unequal(Q, X + Q, E).obstacles == 0
                assert O.filter_unequal(Q, X + Q + Y, E).obstacles == 0
        R = rand_seq(rng, len(Q) + len(Y))
        ham = sum(a != b for a, b in zip(Q, R))
        assert O.filter_unequal(Q, R, 0, stop_above_E=False).obstacles == ham
        assert O.filter_unequal(R, Q, 0, stop_above_E=False).obstacles == ham


def pin_unequal_lower_bound_exhaustive(O):
    """No false reject for approximate string matching: min(count, E+1) never
    exceeds the banded semi-global distance, for every pair of ACGT strings
    of lengths 1..3 and 1..4 that differ, and E <= 2."""
    import itertools
    for mq in range(1, 4):
        for mr in range(1, 5):
            if mq == mr:
                continue
            for q in itertools.product(ALPHA, repeat=mq):
                Q = "".join(q)
                for r in itertools.product(ALPHA, repeat=mr):
                    R = "".join(r)
                    for E in range(3):
                        got = O.filter_unequal(Q, R, E).obstacles
                        assert got <= min(_sg_band(Q, R, E), E + 1), \
                            (Q, R, E, got)


def pin_unequal_optimal(O):
    """Theorem 2 on the corrected maze: the greedy count (routed to the end)
    equals the minimum over every chain of escape segments, by a dynamic
    program over checkpoints on the oracle's own cells."""
    for Q, R in _unequal_pairs(33, 120, 40):
        n = len(R)
        for E in (0, 1, 2, 4):
            Z = [[O.cell2(Q, R, E, i, j) for j in range(1, n + 1)]
                 for i in range(1, 2 * E + 2)]
            inf = 10 ** 9
            best = [inf] * (n + 2)
            best[1] = 0
            for c in range(1, n + 1):
                if best[c] >= inf:
                    continue
                for row in Z:
                    e = c
                    while e <= n and row[e - 1] == 0:
                        e += 1
                    nxt, cost = (n + 1, 0) if e > n else (e + 1, 1)
                    best[nxt] = min(best[nxt], best[c] + cost)
            want = min(best[n + 1:])
            got = O.filter_unequal(Q, R, E, stop_above_E=False).obstacles
            assert got == want, (Q, R, E, got, want)


def pin_unequal_batch_matches_single(O):
    pairs = _unequal_pairs(34, 150, 70)
    reads = "".join(q for q, _ in pairs).encode()
    refs = "".join(r for _, r in pairs).encode()
    rl = np.array([len(q) for q, _ in pairs], np.int32)
    fl = np.array([len(r) for _, r in pairs], np.int32)
    ro = np.concatenate([[0], np.cumsum(rl)[:-1]]).astype(np.int64)
    fo = np.concatenate([[0], np.cumsum(fl)[:-1]]).astype(np.int64)
    Es = np.array([p % 7 for p in range(len(pairs))], np.int32)
    acc, obs = O.filter_unequal_batch(np.frombuffer(reads, np.uint8), ro, rl,
                                      np.frombuffer(refs, np.uint8), fo, fl,
                                      Es, threads=3)
    for p, (Q, R) in enumerate(pairs):
        r = O.filter_unequal(Q, R, int(Es[p]))
        assert (bool(acc[p]), int(obs[p])) == r, p


ALL_PINS = [
    pin_worked_example_maze, pin_worked_example_decision,
    pin_column6_orientation, pin_row_count, pin_identical, pin_E0,
    pin_single_substitution, pin_single_indel, pin_hamming_bound,
    pin_monotone_in_E, pin_cap, pin_cap_counterexample, pin_E_at_least_m,
    pin_optimality, pin_lower_bound_random, pin_lower_bound_exhaustive,
    pin_edit_distance_textbook, pin_edit_distance_bfs, pin_case_and_invalid,
    pin_pack_reference, pin_pack_sliced, pin_batch_matches_single,
    pin_submaze_worked_example, pin_submaze_reduces_to_full,
    pin_submaze_underestimates,
    pin_unequal_equal_lengths_unchanged, pin_unequal_free_flanks,
    pin_unequal_lower_bound_exhaustive, pin_unequal_optimal,
    pin_unequal_batch_matches_single,
]
