"""The oracle's work counters, used for the roofline's op models, against
an independent column-at-a-time walk of the greedy written here in plain
Python (Section 2.4: the AND of the columns from the checkpoint dies at
the column of the longest segment's obstacle)."""
import numpy as np
import pytest

import oracle

CODE = {ord(c): i for i, c in enumerate("ACGT")}


def column_walk(Q: bytes, R: bytes, E: int):
    """(count, columns walked) of the greedy, evaluated column by column."""
    m = len(Q)
    rows = range(-E, E + 1)
    alive = set(rows)
    count = 0
    for j in range(m):
        alive = {s for s in alive if 0 <= j + s < m and Q[j + s] == R[j]}
        if not alive:
            count += 1
            if count > E:
                return count, j + 1
            alive = set(rows)
    return count, m


def test_worked_example_columns():
    res, (cells, words, iters, cols) = oracle.filter_pair(
        b"GGTGAGAGTTGT", b"GGTGCAGAGCTC", 3, with_stats=True)
    assert res.obstacles == 3
    assert cols == 12 and iters == 3  # the third obstacle sits on column 12


@pytest.mark.parametrize("m", [1, 5, 20, 57])
def test_columns_equal_the_column_walk(m):
    rng = np.random.default_rng(m)
    for _ in range(150):
        Q = rng.choice(list(b"ACGT"), m).astype(np.uint8).tobytes()
        R = bytearray(Q)
        for k in rng.integers(0, m, int(rng.integers(0, m // 3 + 2))):
            R[k] = int(rng.choice(list(b"ACGT")))
        R = bytes(R)
        for E in (0, 1, 3, 6):
            res, (_, _, iters, cols) = oracle.filter_pair(Q, R, E,
                                                          with_stats=True)
            count, walked = column_walk(Q, R, E)
            assert min(count, E + 1) == res.obstacles
            assert cols == walked, (Q, R, E)
            assert iters >= min(count, E + 1)


def test_batch_sums_the_counters():
    rng = np.random.default_rng(3)
    reads = rng.choice(list(b"ACGT"), (64, 40)).astype(np.uint8)
    refs = reads.copy()
    refs[::2, 5] = np.where(refs[::2, 5] == ord("A"), ord("C"), ord("A"))
    _, _, tot = oracle.filter_batch(reads, refs, 40, 2, with_stats=True)
    acc = np.zeros(4, np.int64)
    for i in range(64):
        _, st = oracle.filter_pair(reads[i].tobytes(), refs[i].tobytes(), 2,
                                   with_stats=True)
        acc += np.array(st)
    assert tuple(acc) == tuple(tot)
