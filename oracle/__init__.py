"""CPU oracle for the SneakySnake filter (ctypes wrapper of ss_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library; both are fed by the seeded generator in
``paper_1910_09020_gb300.synth``, which holds no filter arithmetic.

Every function follows the paper (Alser et al., SneakySnake):

* :meth:`Oracle.cell`, :meth:`Oracle.maze` -- Eq. 1 (Section 2.3).
* :meth:`Oracle.filter_pair`, :meth:`Oracle.filter_batch` -- the five steps
  of Section 2.4 on the implicit maze; accept = count <= E, obstacles =
  min(count, E+1).
* :meth:`Oracle.min_obstacles` -- the optimum over all chains of escape
  segments (Theorem 2), by dynamic programming over checkpoints.
* :meth:`Oracle.edit_distance` -- textbook Levenshtein DP, the quantity the
  filter bounds from below (Section 2.1).
* :meth:`Oracle.pack_reference` -- the library's documented 2-bit format,
  written from that definition only (checks the pack kernel bit for bit).
* :meth:`Oracle.filter_submaze` -- Snake-on-Chip's sub-maze decomposition
  (Section 2.5).
* :meth:`Oracle.cell2`, :meth:`Oracle.filter_unequal`,
  :meth:`Oracle.filter_unequal_batch` -- pairs of different lengths with the
  leading/trailing case-4 correction of Section 2.4.

Module-level functions call the default instance built from ss_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import NamedTuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "ss_oracle.c")
HEADER = os.path.join(_HERE, "ss_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libss_oracle.so")
_lock = threading.Lock()

OK = 0
ERR_INVALID_ARG = -1
ERR_INVALID_BASE = -2


class Stats(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int64), ("words", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("columns", ctypes.c_int64)]


class Result(NamedTuple):
    accept: bool
    obstacles: int


def compile_oracle(src: str, out: str, include_dir: str = _HERE) -> str:
    """gcc a (possibly modified) copy of the oracle into a shared library."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call([
        "gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-Wall",
        "-fPIC", "-shared", "-pthread", "-I", include_dir, src, "-o", tmp])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + pthreads)."""
    with _lock:
        newest = max(os.path.getmtime(SOURCE), os.path.getmtime(HEADER))
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= newest):
            return _LIB_PATH
        return compile_oracle(SOURCE, _LIB_PATH)


def _bytes(s) -> np.ndarray:
    if isinstance(s, str):
        s = s.encode()
    if isinstance(s, (bytes, bytearray)):
        return np.frombuffer(bytes(s) + b"\0", dtype=np.uint8)
    return np.ascontiguousarray(s, dtype=np.uint8)


def _p(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


class Oracle:
    """One loaded copy of the oracle library."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.sso_cell.argtypes = [P, P, i64, i64, i64, i64]
        lib.sso_cell.restype = ctypes.c_int
        lib.sso_maze.argtypes = [P, P, i64, i64, P]
        lib.sso_filter.argtypes = [P, P, i64, i64, ctypes.c_int, P, P, P]
        lib.sso_min_obstacles.argtypes = [P, P, i64, i64, P]
        lib.sso_filter_submaze.argtypes = [P, P, i64, i64, i64, i64, P, P]
        lib.sso_edit_distance.argtypes = [P, i64, P, i64]
        lib.sso_edit_distance.restype = i64
        lib.sso_filter_batch.argtypes = [P, P, P, P, P, i64, ctypes.c_int,
                                         P, P, P]
        lib.sso_exhaustive_lower_bound.argtypes = [ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, P]
        lib.sso_exhaustive_lower_bound.restype = i64
        lib.sso_pack_reference.argtypes = [P, i64, P]
        lib.sso_pack_sliced.argtypes = [P, i64, i64, P]
        lib.sso_cell2.argtypes = [P, i64, P, i64, i64, i64, i64]
        lib.sso_cell2.restype = ctypes.c_int
        lib.sso_filter2.argtypes = [P, i64, P, i64, i64, ctypes.c_int, P, P]
        lib.sso_filter2_batch.argtypes = [P, P, P, P, P, P, P, i64,
                                          ctypes.c_int, P, P]
        lib.sso_default_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def cell(self, Q, R, E: int, i: int, j: int) -> int:
        """Z[i, j] of Eq. 1, 1-based."""
        q, r = _bytes(Q), _bytes(R)
        return self.lib.sso_cell(_p(q), _p(r), len(Q), E, i, j)

    def maze(self, Q, R, E: int) -> np.ndarray:
        """The complete (2E+1) x m chip maze (Fig. 2b), uint8."""
        q, r = _bytes(Q), _bytes(R)
        m = len(Q)
        Z = np.zeros((2 * E + 1, max(m, 1)), dtype=np.uint8)
        rc = self.lib.sso_maze(_p(q), _p(r), m, E, _p(Z))
        if rc != OK:
            raise ValueError(f"oracle maze error {rc}")
        return Z[:, :m]

    def filter_pair(self, Q, R, E: int, stop_above_E: bool = True,
                    with_stats: bool = False):
        """SneakySnake on one equal-length pair (Section 2.4)."""
        q, r = _bytes(Q), _bytes(R)
        m = len(Q)
        if len(R) != m:
            raise ValueError("pairs must have equal length")
        acc = ctypes.c_uint8()
        obs = ctypes.c_int64()
        st = Stats()
        rc = self.lib.sso_filter(_p(q), _p(r), m, E, int(stop_above_E),
                                 ctypes.byref(acc), ctypes.byref(obs),
                                 ctypes.byref(st))
        if rc != OK:
            raise ValueError(f"oracle filter error {rc}")
        res = Result(bool(acc.value), int(obs.value))
        if with_stats:
            return res, (st.cells, st.words, st.iterations, st.columns)
        return res

    def filter_submaze(self, Q, R, E: int, t: int, y: int) -> Result:
        """Snake-on-Chip decomposition (Section 2.5) into t-column
        sub-mazes, at most y obstacles each."""
        q, r = _bytes(Q), _bytes(R)
        acc = ctypes.c_uint8()
        obs = ctypes.c_int64()
        rc = self.lib.sso_filter_submaze(_p(q), _p(r), len(Q), E, t, y,
                                         ctypes.byref(acc), ctypes.byref(obs))
        if rc != OK:
            raise ValueError(f"oracle submaze error {rc}")
        return Result(bool(acc.value), int(obs.value))

    def cell2(self, Q, R, E: int, i: int, j: int) -> int:
        """Z[i, j] for a query Q and a reference R of any lengths (1-based;
        j indexes R)."""
        q, r = _bytes(Q), _bytes(R)
        return self.lib.sso_cell2(_p(q), len(Q), _p(r), len(R), E, i, j)

    def filter_unequal(self, Q, R, E: int, stop_above_E: bool = True):
        """The filter on a pair of possibly different lengths."""
        q, r = _bytes(Q), _bytes(R)
        acc = ctypes.c_uint8()
        obs = ctypes.c_int64()
        rc = self.lib.sso_filter2(_p(q), len(Q), _p(r), len(R), E,
                                  int(stop_above_E), ctypes.byref(acc),
                                  ctypes.byref(obs))
        if rc != OK:
            raise ValueError(f"oracle filter2 error {rc}")
        return Result(bool(acc.value), int(obs.value))

    def filter_unequal_batch(self, reads, read_off, read_len, refs, ref_off,
                             ref_len, Es, threads: int = 0):
        """Batch of filter_unequal over concatenated byte buffers."""
        reads = np.ascontiguousarray(reads, dtype=np.uint8)
        refs = np.ascontiguousarray(refs, dtype=np.uint8)
        ro = np.ascontiguousarray(read_off, dtype=np.int64)
        rl = np.ascontiguousarray(read_len, dtype=np.int32)
        fo = np.ascontiguousarray(ref_off, dtype=np.int64)
        fl = np.ascontiguousarray(ref_len, dtype=np.int32)
        n = len(rl)
        Es_arr = np.ascontiguousarray(
            np.broadcast_to(np.asarray(Es, np.int32), (n,)))
        acc = np.zeros(max(n, 1), dtype=np.uint8)
        obs = np.zeros(max(n, 1), dtype=np.int32)
        rc = self.lib.sso_filter2_batch(_p(reads), _p(ro), _p(rl), _p(refs),
                                        _p(fo), _p(fl), _p(Es_arr), n,
                                        threads, _p(acc), _p(obs))
        if rc != OK:
            raise ValueError(f"oracle filter2 batch error {rc}")
        return acc[:n], obs[:n]

    def min_obstacles(self, Q, R, E: int) -> int:
        q, r = _bytes(Q), _bytes(R)
        out = ctypes.c_int64()
        rc = self.lib.sso_min_obstacles(_p(q), _p(r), len(Q), E,
                                        ctypes.byref(out))
        if rc != OK:
            raise ValueError(f"oracle min_obstacles error {rc}")
        return int(out.value)

    def edit_distance(self, a, b) -> int:
        x, y = _bytes(a), _bytes(b)
        return int(self.lib.sso_edit_distance(_p(x), len(a), _p(y), len(b)))

    def filter_batch(self, reads: np.ndarray, refs: np.ndarray, lengths, Es,
                     offsets: np.ndarray | None = None, threads: int = 0,
                     with_stats: bool = False):
        """Batch over pairs on host threads.  Fixed-stride form: reads/refs
        of shape (n, m) and offsets None.  Concatenated form: 1-D reads/refs
        with byte offsets (>= n entries) and per-pair lengths."""
        reads = np.ascontiguousarray(reads, dtype=np.uint8)
        refs = np.ascontiguousarray(refs, dtype=np.uint8)
        if offsets is None:
            n = reads.shape[0]
            m = reads.shape[1] if reads.ndim == 2 else int(lengths)
            lens = np.full(max(n, 1), m, dtype=np.int32)
            off = None
        else:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            lens = np.ascontiguousarray(lengths, dtype=np.int32)
            n = len(lens)
        Es_arr = np.ascontiguousarray(
            np.broadcast_to(np.asarray(Es, np.int32), (n,)))
        acc = np.zeros(max(n, 1), dtype=np.uint8)
        obs = np.zeros(max(n, 1), dtype=np.int32)
        st = Stats()
        rc = self.lib.sso_filter_batch(_p(reads), _p(refs), _p(off),
                                       _p(lens), _p(Es_arr), n, threads,
                                       _p(acc), _p(obs), ctypes.byref(st))
        if rc != OK:
            raise ValueError(f"oracle batch error {rc}")
        acc, obs = acc[:n], obs[:n]
        if with_stats:
            return acc, obs, (st.cells, st.words, st.iterations,
                              st.columns)
        return acc, obs

    def batch_status(self, reads, refs, m: int, E: int) -> int:
        """Return code of the batch routine (for invalid-input tests)."""
        reads = np.ascontiguousarray(reads, dtype=np.uint8)
        refs = np.ascontiguousarray(refs, dtype=np.uint8)
        n = reads.shape[0]
        lens = np.full(max(n, 1), m, dtype=np.int32)
        Es = np.full(max(n, 1), E, dtype=np.int32)
        acc = np.zeros(max(n, 1), dtype=np.uint8)
        obs = np.zeros(max(n, 1), dtype=np.int32)
        return self.lib.sso_filter_batch(_p(reads), _p(refs), None, _p(lens),
                                         _p(Es), n, 1, _p(acc), _p(obs), None)

    def exhaustive_lower_bound(self, m: int, Emax: int, threads: int = 0):
        """(violations, pairs) of the lower-bound property over all ACGT
        pairs of length m and every E <= Emax."""
        pairs = ctypes.c_int64()
        v = self.lib.sso_exhaustive_lower_bound(m, Emax, threads,
                                                ctypes.byref(pairs))
        return int(v), int(pairs.value)

    def pack_reference(self, seq) -> np.ndarray:
        s = _bytes(seq)
        m = len(seq)
        out = np.zeros(max((m + 15) // 16, 1), dtype=np.uint32)
        rc = self.lib.sso_pack_reference(_p(s), m, _p(out))
        if rc != OK:
            raise ValueError("invalid base")
        return out[: (m + 15) // 16]

    def pack_sliced(self, seqs: np.ndarray) -> np.ndarray:
        """n sequences of m bases (uint8 array (n, m)) -> the bit-sliced
        layout, 8 * ceil(m/4) * ceil(n/32) uint32 words."""
        s = np.ascontiguousarray(seqs, dtype=np.uint8)
        n, m = s.shape
        out = np.zeros(max(8 * ((m + 3) // 4) * ((n + 31) // 32), 1),
                       dtype=np.uint32)
        rc = self.lib.sso_pack_sliced(_p(s), n, m, _p(out))
        if rc != OK:
            raise ValueError("invalid base")
        return out[: 8 * ((m + 3) // 4) * ((n + 31) // 32)]

    def default_threads(self) -> int:
        return int(self.lib.sso_default_threads())


_default: Oracle | None = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def cell(Q, R, E, i, j):
    return get().cell(Q, R, E, i, j)


def maze(Q, R, E):
    return get().maze(Q, R, E)


def filter_pair(Q, R, E, stop_above_E=True, with_stats=False):
    return get().filter_pair(Q, R, E, stop_above_E, with_stats)


def filter_submaze(Q, R, E, t, y):
    return get().filter_submaze(Q, R, E, t, y)


def min_obstacles(Q, R, E):
    return get().min_obstacles(Q, R, E)


def cell2(Q, R, E, i, j):
    return get().cell2(Q, R, E, i, j)


def filter_unequal(Q, R, E, stop_above_E=True):
    return get().filter_unequal(Q, R, E, stop_above_E)


def filter_unequal_batch(reads, read_off, read_len, refs, ref_off, ref_len,
                         Es, threads=0):
    return get().filter_unequal_batch(reads, read_off, read_len, refs,
                                      ref_off, ref_len, Es, threads)


def edit_distance(a, b):
    return get().edit_distance(a, b)


def filter_batch(reads, refs, lengths, Es, offsets=None, threads=0,
                 with_stats=False):
    return get().filter_batch(reads, refs, lengths, Es, offsets, threads,
                              with_stats)


def pack_reference(seq):
    return get().pack_reference(seq)


def pack_sliced(seqs):
    return get().pack_sliced(seqs)


def default_threads():
    return get().default_threads()
