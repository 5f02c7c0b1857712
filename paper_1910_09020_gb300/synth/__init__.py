"""Seeded synthetic read/reference pairs shaped like the paper's workloads.

This module draws random sequences and random edits only; it contains none of
the filter's arithmetic, so the CUDA path and the CPU oracle can both be fed
from it.  Each pair comes from its own counter-based stream keyed by (seed,
pair index): any subset of a workload can be regenerated on its own.

Workload shapes (SneakySnake, Section 3.1 and the configurations measured
here):

* ``short_uniform_k``   100 bp, k ~ U{0..10} edits, types equiprobable.
* ``short_poisson``     100 bp; even pairs carry Poisson(3) edits (types
                         equiprobable), odd pairs are independent random
                         sequences (the "_2"-style dissimilar half).
* ``rate``              per-pair edit rate r ~ U[0, rmax]; each read base is
                         edited with probability r; substitution 80 %,
                         insertion 10 %, deletion 10 %.

The reference segment is always cut or padded with random bases back to the
read's length (equal-length pairs, Section 2.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None

MODE_UNIFORM_K = 0
MODE_POISSON = 1
MODE_RATE = 2


class _Params(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32),
        ("kmin", ctypes.c_int32),
        ("kmax", ctypes.c_int32),
        ("lam", ctypes.c_double),
        ("rmax", ctypes.c_double),
        ("psub", ctypes.c_double),
        ("pins", ctypes.c_double),
        ("pdel", ctypes.c_double),
    ]


@dataclass(frozen=True)
class Recipe:
    """How the reference segment is derived from the read."""

    mode: int
    kmin: int = 0
    kmax: int = 0
    lam: float = 0.0
    rmax: float = 0.0
    psub: float = 1.0
    pins: float = 1.0
    pdel: float = 1.0

    def _c(self) -> _Params:
        return _Params(self.mode, self.kmin, self.kmax, self.lam, self.rmax,
                       self.psub, self.pins, self.pdel)


SHORT_UNIFORM_K = Recipe(MODE_UNIFORM_K, kmin=0, kmax=10)
SHORT_POISSON = Recipe(MODE_POISSON, lam=3.0)


def rate_recipe(rmax: float) -> Recipe:
    return Recipe(MODE_RATE, rmax=rmax, psub=0.8, pins=0.1, pdel=0.1)


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library next to this file."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-fPIC",
            "-shared", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.synth_pairs.argtypes = [
            ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
            P, P, ctypes.POINTER(_Params), P, P, ctypes.c_int]
        lib.synth_log_uniform.argtypes = [
            ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
            ctypes.c_double, ctypes.c_uint64, P]
        lib.synth_poisson_arrivals.argtypes = [
            ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def pairs_fixed(seed: int, first: int, n: int, m: int, recipe: Recipe,
                threads: int = 0, out: tuple | None = None):
    """n pairs of length m: returns (reads, refs), uint8 arrays of shape
    (n, m), ASCII upper-case ACGT.  Pass ``out`` to fill existing arrays
    (e.g. pinned host tensors viewed as numpy)."""
    lib = _load()
    if out is None:
        reads = np.empty((n, m), dtype=np.uint8)
        refs = np.empty((n, m), dtype=np.uint8)
    else:
        reads, refs = out
        assert reads.dtype == np.uint8 and reads.size >= n * m
        assert refs.dtype == np.uint8 and refs.size >= n * m
        assert reads.flags.c_contiguous and refs.flags.c_contiguous
    p = recipe._c()
    lib.synth_pairs(seed, first, n, m, None, None, ctypes.byref(p),
                    _ptr(reads), _ptr(refs), threads)
    return reads, refs


def offsets_of(lengths: np.ndarray) -> np.ndarray:
    """Byte offsets (n+1 entries) of concatenated sequences."""
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def pairs_varlen(seed: int, first: int, lengths: np.ndarray, recipe: Recipe,
                 threads: int = 0):
    """Pairs with per-pair lengths, concatenated: returns (reads, refs,
    offsets) with offsets of length n+1 (bytes)."""
    lib = _load()
    lengths = np.ascontiguousarray(lengths, dtype=np.int32)
    off = offsets_of(lengths)
    total = int(off[-1])
    reads = np.empty(max(total, 1), dtype=np.uint8)
    refs = np.empty(max(total, 1), dtype=np.uint8)
    p = recipe._c()
    lib.synth_pairs(seed, first, len(lengths), 0, _ptr(off), _ptr(lengths),
                    ctypes.byref(p), _ptr(reads), _ptr(refs), threads)
    return reads[:total], refs[:total], off


def log_uniform(seed: int, first: int, n: int, lo: float, hi: float,
                salt: int = 0x1E9) -> np.ndarray:
    """floor(exp(U[ln lo, ln hi])) per index, int32."""
    lib = _load()
    out = np.empty(n, dtype=np.int32)
    lib.synth_log_uniform(seed, first, n, float(lo), float(hi), salt,
                          _ptr(out))
    return out


def poisson_arrivals(seed: int, n: int, rate: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    lib = _load()
    out = np.empty(n, dtype=np.float64)
    lib.synth_poisson_arrivals(seed, n, float(rate), _ptr(out))
    return out


def thresholds(lengths: np.ndarray, percent: float) -> np.ndarray:
    """E = floor(percent * m / 100) per pair (a threshold given as a share of
    the read length)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    # integer arithmetic on percent * 1000 keeps floor() exact
    num = lengths * int(round(percent * 1000))
    return (num // 100000).astype(np.int32)


def pairs_unequal(seed: int, first: int, n: int, m: int, recipe: Recipe,
                  delta_lo: int, delta_hi: int, threads: int = 0):
    """Reads of m bases against reference windows of m + d bases, d uniform
    in delta_lo..delta_hi per pair: for d >= 0 the window is the edited copy
    of the read with random flanks of o and d - o bases (o uniform in
    0..d); for d < 0 it is the edited copy cut to m + d bases.  Returns
    (reads, read_offsets, read_lengths, refs, ref_offsets, ref_lengths),
    offsets in bytes (n + 1 entries)."""
    core_len = np.full(n, m, dtype=np.int32)
    reads, core, _ = pairs_varlen(seed, first, core_len, recipe, threads)
    core = core[:n * m].reshape(n, m) if m > 0 else core[:0].reshape(n, 0)
    rng = np.random.default_rng([seed, first, n, 0x0E0A1])
    d = rng.integers(delta_lo, delta_hi + 1, size=n)
    o = (rng.random(n) * (np.maximum(d, 0) + 1)).astype(np.int64)
    ref_len = np.maximum(m + d, 0).astype(np.int32)
    ref_off = offsets_of(ref_len)
    total = int(ref_off[-1])
    alphabet = np.frombuffer(b"ACGT", dtype=np.uint8)
    refs = alphabet[rng.integers(0, 4, size=max(total, 1), dtype=np.uint8)]
    col = np.arange(m, dtype=np.int64)
    chunk = max(1, (1 << 24) // max(m, 1))
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        start = ref_off[a:b] + np.where(d[a:b] >= 0, o[a:b], 0)
        keep = col[None, :] < ref_len[a:b, None]  # d < 0: cut the tail
        idx = start[:, None] + col[None, :]
        refs[idx[keep]] = core[a:b][keep]
    return (reads, offsets_of(core_len), core_len, refs[:total], ref_off,
            ref_len)
