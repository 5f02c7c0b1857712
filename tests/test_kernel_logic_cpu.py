"""The library's routing functions, compiled for the host by the test
harness in tests/kernel_emu, against the CPU oracle (no GPU needed).

This checks the kernels' logic (word crossings, edge masks, runtime
thresholds, the column-wise phases) quickly on the CPU; the GPU parity
tests remain the proof that the kernels themselves agree with the oracle.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1910_09020_gb300 import synth

kernel_emu = pytest.importorskip("kernel_emu")


@pytest.fixture(scope="module")
def emu():
    return kernel_emu.load()


def packed(seq: bytes) -> np.ndarray:
    w = oracle.pack_reference(seq)
    return np.concatenate([w, np.zeros(2, np.uint32)])  # slack for reads


def P(a):
    return ctypes.c_void_p(a.ctypes.data)


def pairs(seed, n, m, recipe):
    r, f = synth.pairs_fixed(seed, 0, n, m, recipe)
    return [(r[i].tobytes(), f[i].tobytes()) for i in range(n)]


@pytest.mark.parametrize("m", [1, 2, 17, 31, 32, 33, 64, 65, 100, 150, 257])
def test_rw_exact_matches_oracle(emu, m):
    for Q, R in pairs(60 + m, 60, m, synth.rate_recipe(0.15)):
        q, r = packed(Q), packed(R)
        for E in (0, 1, 2, 3, 4, 5, 10, 17, 31):
            got = emu.emu_rw_exact(P(q), P(r), m, E)
            want = oracle.filter_pair(Q, R, E).obstacles
            assert got == want, (m, E, Q, R)


@pytest.mark.parametrize("m", [1, 2, 7, 8, 9, 15, 16, 17, 31, 32, 33, 40,
                               64, 65, 100, 150, 250, 257])
def test_rw_cols_matches_oracle(emu, m):
    """Column-at-a-time routine: every E it supports (one survivor word to
    E = 15, two from 16 to 31), lengths around the 8-column chunks and
    32-column words, edges on both sides."""
    for Q, R in pairs(1700 + m, 40, m, synth.rate_recipe(0.12)):
        q, r = packed(Q), packed(R)
        for E in range(1, 32):
            got = emu.emu_rw_cols(P(q), P(r), m, E)
            want = oracle.filter_pair(Q, R, E).obstacles
            assert got == want, (m, E, Q, R)


def test_rw_cols_headline_recipe(emu):
    """The headline workload's pairs (Poisson(3) edits or random) at the
    sweep's thresholds."""
    reads, refs = synth.pairs_fixed(5, 0, 400, 100, synth.SHORT_POISSON)
    for i in range(400):
        Q, R = reads[i].tobytes(), refs[i].tobytes()
        q, r = packed(Q), packed(R)
        for E in (2, 4, 5, 6, 8, 10, 15, 16, 20, 31):
            assert emu.emu_rw_cols(P(q), P(r), 100, E) == \
                oracle.filter_pair(Q, R, E).obstacles, (i, E)


@pytest.mark.parametrize("emax", [1, 3, 7, 15, 31])
def test_rw_runtime_threshold_matches_oracle(emu, emax):
    rng = np.random.default_rng(emax)
    for i in range(150):
        m = int(rng.integers(1, 400))
        Q, R = pairs(900 + i, 1, m, synth.rate_recipe(0.12))[0]
        q, r = packed(Q), packed(R)
        E = int(rng.integers(0, emax + 1))
        if rng.random() < 0.2:
            E = m + int(rng.integers(0, 5))  # E >= m (rows clamped)
            if min(E, m - 1) > emax:
                continue
        got = emu.emu_rw_runtime(P(q), P(r), m, E, emax)
        want = oracle.filter_pair(Q, R, E).obstacles
        assert got == want, (m, E, emax)


@pytest.mark.parametrize("K", [4, 8, 16])
def test_cw_matches_oracle(emu, K):
    rng = np.random.default_rng(K)
    for i in range(60):
        m = int(np.exp(rng.uniform(np.log(2), np.log(2500))))
        E = int(rng.choice([0, 3, 31, 32, 70, m // 10, m // 2, m + 3]))
        rec = synth.rate_recipe(float(rng.choice([0.01, 0.05, 0.2])))
        Q, R = pairs(500 + i, 1, m, rec)[0]
        q, r = packed(Q), packed(R)
        got = emu.emu_cw(P(q), P(r), m, E, K)
        want = oracle.filter_pair(Q, R, E).obstacles
        assert got == want, (m, E, K)


def test_worked_example_every_routine(emu):
    Q, R = b"GGTGAGAGTTGT", b"GGTGCAGAGCTC"
    q, r = packed(Q), packed(R)
    assert emu.emu_rw_exact(P(q), P(r), 12, 3) == 3
    assert emu.emu_rw_runtime(P(q), P(r), 12, 3, 7) == 3
    for K in (4, 8, 16):
        assert emu.emu_cw(P(q), P(r), 12, 3, K) == 3


def test_class_table_covers_the_shapes(emu):
    seen = set()
    for m, E in [(100, 0), (100, 3), (100, 7), (100, 15), (100, 31),
                 (1000, 50), (5000, 250), (12000, 500), (20000, 40),
                 (3000, 600), (50000, 5000), (100000, 10000), (131072, 100)]:
        c = emu.emu_class_of(m, E)
        assert c >= 0, (m, E)
        seen.add(c)
    assert len(seen) >= 10
    assert emu.emu_class_of(0, 5) == -1
    assert emu.emu_class_of(5, -1) == -2
    assert emu.emu_class_of(200000, 500) == -3
    assert emu.emu_class_of(200000, 20) == 4  # small E: any length


@pytest.mark.parametrize("m", [1, 5, 16, 17, 40, 100, 150])
def test_banded_edit_distance_matches_oracle(emu, m):
    """Accuracy-harness verifier: min(ED, E+1) against the oracle's DP."""
    for Q, R in pairs(700 + m, 40, m, synth.rate_recipe(0.2)):
        q, r = packed(Q), packed(R)
        ed = oracle.edit_distance(Q, R)
        for E in (0, 1, 2, 5, 10, 20, 31):
            assert emu.emu_ed(P(q), P(r), m, E) == min(ed, E + 1), (m, E)


@pytest.mark.parametrize("t", [1, 3, 8, 31, 32, 33, 77, 1000])
def test_submaze_matches_oracle(emu, t):
    """The kernel's choice and both sub-maze routines (the column walk at
    every class up to E' = 15, the row-wise one at every class) against
    the oracle."""
    rng = np.random.default_rng(t)
    for i in range(40):
        m = int(rng.integers(1, 180))
        Q, R = pairs(800 + i, 1, m, synth.rate_recipe(0.12))[0]
        q, r = packed(Q), packed(R)
        for E in (0, 1, 2, 5, 9, 15, 20, 31):
            for y in (1, 3, 1000):
                want = oracle.filter_submaze(Q, R, E, t, y).obstacles
                got = emu.emu_submaze(P(q), P(r), m, E, t, y)
                assert got == want, (m, E, t, y)
                got = emu.emu_submaze_rows(P(q), P(r), m, E, t, y)
                assert got == want, ("rows", m, E, t, y)
                got = emu.emu_submaze_cols(P(q), P(r), m, E, t, y)
                assert got in (want, -2), ("cols", m, E, t, y)


@pytest.mark.parametrize("m", [1, 7, 16, 17, 31, 32, 33, 63, 64, 65, 100,
                               127, 128, 150, 200, 256])
def test_staged_reads_ignore_what_follows(emu, m):
    """The pipelined kernels route a pair in place in its shared-memory
    stage, where the words after it are the next pair's (or the tile's R
    words): the plain and sub-maze routines must give the oracle's result
    whatever those words hold."""
    rng = np.random.default_rng(m)
    w16 = (m + 15) // 16

    def staged(seq):
        junk = rng.integers(0, 2**32, 8, dtype=np.uint64).astype(np.uint32)
        return np.concatenate([oracle.pack_reference(seq)[:w16], junk])

    for Q, R in pairs(2100 + m, 10, m, synth.rate_recipe(0.12)):
        q, r = staged(Q), staged(R)
        for E in range(32):
            want = oracle.filter_pair(Q, R, E).obstacles
            assert emu.emu_rw_staged(P(q), P(r), m, E, 0) == want, (m, E)
            if 1 <= E <= 31:
                got = emu.emu_rw_staged(P(q), P(r), m, E, 1)
                assert got == want, ("cols", m, E)
        for E in (0, 2, 5, 9, 15, 31):
            for t in (5, 8, 32):
                for y in (1, 3):
                    want = oracle.filter_submaze(Q, R, E, t, y).obstacles
                    for form in (0, 1, 2):
                        got = emu.emu_submaze_staged(P(q), P(r), m, E, t, y,
                                                     form)
                        assert got == want or (form == 2 and got == -2), (
                            m, E, t, y, form)


CODE = {c: i for i, c in enumerate(b"ACGT")}
CODE.update({c: i for i, c in enumerate(b"acgt")})


def test_pack_chunk_every_byte_value_every_position(emu):
    """Validity rule and code gather of the pack kernels on all 256 byte
    values at each of the 16 positions, against the oracle's packer."""
    err = ctypes.c_uint32()
    for pos in range(16):
        for b in range(256):
            buf = bytearray(b"A" * 16)
            buf[pos] = b
            arr = np.frombuffer(bytes(buf), np.uint8).copy()
            got = emu.emu_pack_chunk(P(arr), ctypes.byref(err))
            assert (err.value == 0) == (b in CODE), (pos, b)
            if b in CODE:
                assert got == int(oracle.pack_reference(bytes(buf))[0]), (pos, b)


def pair_order(packed_word: int) -> int:
    """The oracle's 2-bit word (bit t: code bit 0, bit 16+t: code bit 1)
    rearranged to base order: base t at bits 2t and 2t+1."""
    out = 0
    for t in range(16):
        out |= ((packed_word >> t) & 1) << (2 * t)
        out |= ((packed_word >> (16 + t)) & 1) << (2 * t + 1)
    return out


def test_pack_chunk_pairs_every_byte_value_every_position(emu):
    """The sliced packer's arithmetic (code bits in base order) on all 256
    byte values at each of the 16 positions, against the oracle's packer."""
    err = ctypes.c_uint32()
    for pos in range(16):
        for b in range(256):
            buf = bytearray(b"A" * 16)
            buf[pos] = b
            arr = np.frombuffer(bytes(buf), np.uint8).copy()
            got = emu.emu_pack_chunk_pairs(P(arr), ctypes.byref(err))
            assert (err.value == 0) == (b in CODE), (pos, b)
            if b in CODE:
                want = pair_order(int(oracle.pack_reference(bytes(buf))[0]))
                assert got == want, (pos, b)
    rng = np.random.default_rng(4)
    for _ in range(300):
        s = rng.choice(list(b"ACGTacgt"), 16).astype(np.uint8).tobytes()
        arr = np.frombuffer(s, np.uint8).copy()
        got = emu.emu_pack_chunk_pairs(P(arr), ctypes.byref(err))
        assert err.value == 0
        assert got == pair_order(int(oracle.pack_reference(s)[0]))


def test_pack_chunk_and_window_random_streams(emu):
    rng = np.random.default_rng(3)
    err = ctypes.c_uint32()
    for _ in range(200):
        s = rng.choice(list(b"ACGTacgt"), 64).astype(np.uint8).tobytes()
        arr = np.frombuffer(s, np.uint8).copy()
        chunks = []
        for k in range(4):
            sub = arr[16 * k:16 * k + 16].copy()
            w = emu.emu_pack_chunk(P(sub), ctypes.byref(err))
            assert err.value == 0
            assert w == int(oracle.pack_reference(s[16 * k:16 * k + 16])[0])
            chunks.append(w)
        for k in range(3):
            for r in range(16):
                got = emu.emu_pack_window(chunks[k], chunks[k + 1], r)
                start = 16 * k + r
                assert got == int(oracle.pack_reference(s[start:start + 16])[0])


def test_unequal_lengths_match_oracle(emu):
    """Pairs of different lengths (and some equal): the library's routine
    against oracle.filter_unequal."""
    rng = np.random.default_rng(11)
    for i in range(400):
        mq = int(rng.integers(1, 300))
        mr = max(1, mq + int(rng.choice([-40, -9, -3, -1, 0, 1, 2, 5, 17, 70])))
        rec = synth.rate_recipe(float(rng.choice([0.02, 0.1, 0.3])))
        Q, R = pairs(1200 + i, 1, max(mq, mr), rec)[0]
        Q = Q[:mq]
        R = R[:mr]
        q, r = packed(Q), packed(R)
        for E in (0, 1, 2, 3, 5, 7, 9, 12, 15, 20, 31):
            want = oracle.filter_unequal(Q, R, E).obstacles
            got = emu.emu_unequal(P(q), mq, P(r), mr, E)
            assert got in (want, -2), (mq, mr, E, got, want)
            for form in (0, 1):  # row-wise and column walk, every class
                got = emu.emu_unequal_form(P(q), mq, P(r), mr, E, form)
                assert got in (want, -2), (form, mq, mr, E, got, want)


def test_unequal_exact_threshold_routines_match_oracle(emu):
    """The uniform-threshold launch's routine for every E from 0 to 31
    (row-wise, the frame-form column walk from 5 to 14, the shifted-window
    walk at 15), on pairs of different and equal lengths around the 8-column
    chunks, the 32-column words and the ends."""
    rng = np.random.default_rng(13)
    for i in range(160):
        mq = int(rng.integers(1, 300))
        mr = max(1, mq + int(rng.choice([-40, -9, -3, -1, 0, 1, 2, 5, 17, 70])))
        rec = synth.rate_recipe(float(rng.choice([0.02, 0.1, 0.3])))
        Q, R = pairs(4100 + i, 1, max(mq, mr), rec)[0]
        Q, R = Q[:mq], R[:mr]
        q, r = packed(Q), packed(R)
        for E in range(32):
            want = oracle.filter_unequal(Q, R, E).obstacles
            got = emu.emu_unequal_exact(P(q), mq, P(r), mr, E)
            assert got == want, (mq, mr, E, got, want)


def test_unequal_staged_reads_ignore_what_follows(emu):
    """The unequal-length tile kernel routes a pair in place in its
    shared-memory slot, where the words after its sequences are another
    pair's (or leftovers): the routine of each row class must give the
    oracle's result whatever those words hold, at lengths to 256."""
    rng = np.random.default_rng(12)

    def slot(seq):
        w = (len(seq) + 15) // 16
        junk = rng.integers(0, 2**32, 8, dtype=np.uint64).astype(np.uint32)
        return np.concatenate([oracle.pack_reference(seq)[:w], junk])

    for i in range(240):
        mq = int(rng.integers(1, 257))
        mr = int(min(256, max(1, mq + rng.choice([-20, -5, -1, 0, 3, 9, 16]))))
        rec = synth.rate_recipe(float(rng.choice([0.02, 0.1, 0.3])))
        Q, R = pairs(3100 + i, 1, max(mq, mr), rec)[0]
        Q, R = Q[:mq], R[:mr]
        q, r = slot(Q), slot(R)
        for E in (0, 2, 3, 5, 7, 10, 15, 16, 31):
            want = oracle.filter_unequal(Q, R, E).obstacles
            got = emu.emu_unequal_staged(P(q), mq, P(r), mr, E)
            assert got in (want, -2), (mq, mr, E, got, want)


@pytest.mark.parametrize("K", [4, 8, 16])
def test_cw_long_reads_match_oracle(emu, K):
    """Column-wise routine on long reads at E = 10 % of the length: edge
    and interior row words, survivors past K columns (low edit rates) and
    both blocks of the 16-column phase."""
    rng = np.random.default_rng(40 + K)
    for i in range(6):
        m = int(rng.integers(3000, 8000))
        E = m // 10
        rec = synth.rate_recipe(float(rng.choice([0.003, 0.02, 0.08, 0.15])))
        Q, R = pairs(1500 + i, 1, m, rec)[0]
        q, r = packed(Q), packed(R)
        got = emu.emu_cw(P(q), P(r), m, E, K)
        want = oracle.filter_pair(Q, R, E).obstacles
        assert got == want, (m, E, K)


def test_sliced_transpose_is_the_bit_transpose(emu):
    """The sliced packer's warp transpose (32 lanes simulated): lane r ends
    with bit r of every lane's word, bit i from lane i."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        v = rng.integers(0, 2**32, 32, dtype=np.uint64).astype(np.uint32)
        out = np.zeros(32, np.uint32)
        emu.emu_transpose32(P(v), P(out))
        bits = (v[:, None] >> np.arange(32, dtype=np.uint32)) & 1  # [i][r]
        want = (bits.T.astype(np.uint64) << np.arange(32, dtype=np.uint64)
                ).sum(axis=1).astype(np.uint32)
        assert (out == want).all()


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7, 9, 15, 16, 31, 33, 64, 100,
                               101, 150, 251])
def test_sliced_walk_matches_oracle(emu, m):
    """The bit-sliced walk (32 pairs per thread, columns in blocks of four,
    the query window either side, the thermometer count below E = 11 and
    the saturating binary count from it) at every E it is built for, on groups
    mixing near and far pairs, a ragged last group, lengths below, at and
    around E and the block edges."""
    rng = np.random.default_rng(1000 + m)
    n = int(rng.choice([1, 31, 32, 33, 95]))
    rec = synth.rate_recipe(float(rng.choice([0.03, 0.12, 0.4])))
    reads, refs = synth.pairs_fixed(7000 + m, 0, n, m, rec)
    q = oracle.pack_sliced(reads)
    r = oracle.pack_sliced(refs)
    for E in range(32):
        acc = np.zeros(n, np.uint8)
        obs = np.zeros(n, np.int32)
        assert emu.emu_sliced(P(q), P(r), n, m, E, P(acc), P(obs)) == 0
        oacc, oobs = oracle.filter_batch(reads, refs, m, E)
        bad = np.flatnonzero((acc != oacc) | (obs != oobs))
        assert bad.size == 0, (m, n, E, bad[:5], obs[bad[:5]], oobs[bad[:5]])


# (read length, reference length): references longer and shorter, by less
# and more than E, around the block edges, a one-base sequence
FREE_SHAPES = [(100, 116), (100, 92), (100, 101), (100, 99), (33, 40),
               (40, 33), (5, 9), (9, 5), (1, 4), (4, 1), (16, 17), (150, 100)]


@pytest.mark.parametrize("mq,mr", FREE_SHAPES)
def test_sliced_free_walk_matches_oracle(emu, mq, mr):
    """The sliced walk over the reference's columns against a read of
    another length, with Section 2.4's correction (cells past either end of
    the read free), at every E it is built for, against the oracle's
    sso_filter2 pair by pair: reads inside flanked windows, cut windows and
    unrelated pairs, a ragged last group."""
    rng = np.random.default_rng(3000 + 7 * mq + mr)
    n = 70
    reads, _ = synth.pairs_fixed(7200 + mq, 0, n, mq, synth.rate_recipe(0.1))
    refs = synth.pairs_fixed(7300 + mr, 0, n, mr, synth.SHORT_POISSON)[1]
    # half the references: the read itself inside random flanks (or cut)
    for p in range(0, n, 2):
        o = int(rng.integers(0, max(mr - mq, 0) + 1))
        k = min(mq, mr - o)
        refs[p, o:o + k] = reads[p, :k]
    q = oracle.pack_sliced(reads)
    r = oracle.pack_sliced(refs)
    ro = np.arange(n + 1, dtype=np.int64) * mq
    fo = np.arange(n + 1, dtype=np.int64) * mr
    for E in range(32):
        acc = np.zeros(n, np.uint8)
        obs = np.zeros(n, np.int32)
        assert emu.emu_sliced_free(P(q), P(r), n, mq, mr, E, P(acc),
                                   P(obs)) == 0
        oacc, oobs = oracle.filter_unequal_batch(
            reads.reshape(-1), ro[:-1], np.full(n, mq, np.int32),
            refs.reshape(-1), fo[:-1], np.full(n, mr, np.int32), E)
        bad = np.flatnonzero((acc != oacc) | (obs != oobs))
        assert bad.size == 0, (mq, mr, E, bad[:5], obs[bad[:5]],
                               oobs[bad[:5]])


SETS = {0: (0, 2, 4), 1: (0, 1, 2, 3, 4), 2: (1, 3), 3: (3, 4)}


@pytest.mark.parametrize("m", [1, 3, 5, 9, 16, 33, 100, 150])
def test_sliced_threshold_sets_match_oracle(emu, m):
    """Several thresholds walked in one pass over the sliced layout (one
    window for the largest, each its own rows and count): every threshold's
    results equal the oracle's, groups ragged."""
    rng = np.random.default_rng(2000 + m)
    n = int(rng.choice([7, 32, 70]))
    reads, refs = synth.pairs_fixed(7100 + m, 0, n, m, synth.rate_recipe(0.1))
    q, r = oracle.pack_sliced(reads), oracle.pack_sliced(refs)
    for which, Es in SETS.items():
        accs = [np.zeros(n, np.uint8) for _ in Es]
        obss = [np.zeros(n, np.int32) for _ in Es]
        pa = (ctypes.c_void_p * len(Es))(*[a.ctypes.data for a in accs])
        po = (ctypes.c_void_p * len(Es))(*[o.ctypes.data for o in obss])
        assert emu.emu_sliced_set(P(q), P(r), n, m, which, pa, po) == 0
        for i, E in enumerate(Es):
            oacc, oobs = oracle.filter_batch(reads, refs, m, E)
            assert (accs[i] == oacc).all() and (obss[i] == oobs).all(), \
                (m, Es, E)


@pytest.mark.parametrize("m", [1, 5, 8, 9, 17, 64, 100, 150])
def test_sliced_submaze_matches_oracle(emu, m):
    """The sub-maze mode on the sliced walk (every row restarting at each
    sub-maze's first column, at most y counted segments per sub-maze): the
    oracle's sso_filter_submaze at widths within, at and around the
    4-column blocks, y from 1 to beyond E+1, E up to 15."""
    rng = np.random.default_rng(3000 + m)
    n = int(rng.choice([9, 33, 64]))
    reads, refs = synth.pairs_fixed(7200 + m, 0, n, m, synth.rate_recipe(0.15))
    q, r = oracle.pack_sliced(reads), oracle.pack_sliced(refs)
    for E in (0, 1, 3, 6, 10, 15):
        for t, y in ((1, 1), (3, 2), (4, 1), (8, 3), (13, 2), (1000, 99)):
            acc = np.zeros(n, np.uint8)
            obs = np.zeros(n, np.int32)
            assert emu.emu_sliced_submaze(P(q), P(r), n, m, E, t, y, P(acc),
                                          P(obs)) == 0
            for p in range(n):
                want = oracle.filter_submaze(reads[p].tobytes(),
                                             refs[p].tobytes(), E, t, y)
                assert (bool(acc[p]), int(obs[p])) == \
                    (want.accept, want.obstacles), (m, E, t, y, p)
