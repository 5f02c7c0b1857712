"""Thin ctypes binding of the C ABI in ``include/ss.h``.

Argument marshalling only: every step of the filter runs in the CUDA
library.  The functions below carry the C names (``ss_create``,
``ss_filter_batch`` ...) and take plain integers for pointers;
:class:`Filter` adds the marshalling of torch tensors (``data_ptr()``,
current CUDA stream).  Loading raises if the library cannot be built or
loaded -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

from . import build as _build

SS_OK = 0
SS_ERR_INVALID_ARG = -1
SS_ERR_INVALID_BASE = -2
SS_ERR_OOM = -3
SS_ERR_CUDA = -4
SS_ERR_TIMEOUT = -5
SS_ERR_BUSY = -6
SS_ERR_UNSUPPORTED = -7

SS_FMT_ASCII = 0
SS_FMT_PACKED2 = 1
SS_FMT_SLICED2 = 2

SS_MODE_AUTO = 0
SS_MODE_PLAIN = 1
SS_MODE_BUCKETED = 2
SS_FLAG_NO_GRAPH = 16

# largest uniform E and m the plain launch covers (SS_PLAIN_MAX_E/_M)
PLAIN_MAX_E = 31
PLAIN_MAX_M = 1024
# largest E of the plain launch over SS_FMT_SLICED2 input (SS_SLICED_MAX_E)
SLICED_MAX_E = 31

# every symbol include/ss.h declares (checked by the CPU tests)
EXPORTED = (
    "ss_create", "ss_destroy", "ss_strerror", "ss_version",
    "ss_packed_words", "ss_pack", "ss_filter_batch", "ss_filter_host",
    "ss_sliced_words", "ss_pack_sliced", "ss_filter_sweep",
    "ss_filter_segments",
    "ss_sync", "ss_get_counters", "ss_set_tuning", "ss_get_tuning",
    "ss_autotune", "ss_filter_batch_noalloc", "ss_edit_distance_banded",
    "ss_filter_confusion", "ss_compact_accepted", "ss_gather_pairs",
    "ss_filter_submaze", "ss_check_wait_timeout", "ss_filter_unequal",
    "ss_edit_distance_varlen",
    "ss_server_create",
    "ss_server_submit", "ss_server_poll", "ss_server_wait", "ss_server_fetch",
    "ss_server_get_stats", "ss_server_reset_stats", "ss_server_destroy",
)
SS_NOALLOC_MAX_PAIRS = 1048576


class SSError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class ServerStats(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_int64),
                ("pairs_done", ctypes.c_int64),
                ("bases_done", ctypes.c_int64),
                ("batches", ctypes.c_int64),
                ("max_inflight", ctypes.c_int64),
                ("pending", ctypes.c_int64),
                ("device_bytes_in_use", ctypes.c_int64),
                ("latency_p50_s", ctypes.c_double),
                ("latency_p99_s", ctypes.c_double),
                ("latency_max_s", ctypes.c_double),
                ("span_s", ctypes.c_double),
                ("long_pairs_queued", ctypes.c_int64),
                ("worker_launches", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Segment(ctypes.Structure):
    """ss_segment: one uniform batch of ss_filter_segments."""
    _fields_ = [("reads", ctypes.c_void_p), ("refs", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("m", ctypes.c_int32),
                ("e", ctypes.c_int32), ("out_accept", ctypes.c_void_p),
                ("out_obstacles", ctypes.c_void_p), ("m_ref", ctypes.c_int32)]


class Counters(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libss.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library not built: {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    P, I32, I64, SZ = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                       ctypes.c_size_t)
    lib.ss_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, SZ]
    lib.ss_destroy.argtypes = [P]
    lib.ss_strerror.argtypes = [ctypes.c_int]
    lib.ss_strerror.restype = ctypes.c_char_p
    lib.ss_version.restype = ctypes.c_int
    lib.ss_packed_words.argtypes = [I64]
    lib.ss_packed_words.restype = I64
    lib.ss_pack.argtypes = [P, P, P, P, I32, I64, P, P, P]
    lib.ss_sliced_words.argtypes = [I64, I64]
    lib.ss_sliced_words.restype = I64
    lib.ss_pack_sliced.argtypes = [P, P, I32, I64, P, P]
    lib.ss_filter_sweep.argtypes = [P, P, P, ctypes.c_int, I32, P,
                                    ctypes.c_int, I64, P, P, P]
    lib.ss_filter_segments.argtypes = [P, ctypes.POINTER(Segment),
                                       ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, P]
    lib.ss_filter_batch.argtypes = [P, P, P, ctypes.c_int, P, P, I32, P, I32,
                                    I64, ctypes.c_int, P, P, P]
    lib.ss_filter_host.argtypes = [P, P, P, ctypes.c_int, I32, P,
                                   ctypes.c_int, I64, P, P]
    lib.ss_sync.argtypes = [P, P]
    lib.ss_get_counters.argtypes = [P, ctypes.POINTER(Counters)]
    lib.ss_filter_batch_noalloc.argtypes = [P, P, P, P, I32, P, I32, I64, P,
                                            P, P]
    lib.ss_edit_distance_banded.argtypes = [P, P, P, ctypes.c_int, I32, I32,
                                            I64, P, P]
    lib.ss_filter_confusion.argtypes = [P, P, P, I64, I32, P, P]
    lib.ss_compact_accepted.argtypes = [P, P, I64, P, P, P]
    lib.ss_check_wait_timeout.argtypes = [P, I64, P]
    lib.ss_edit_distance_varlen.argtypes = [P, P, P, P, P, P, I64, P, P]
    lib.ss_filter_unequal.argtypes = [P, P, P, P, P, P, P, P, I32, I64, P,
                                      P, P]
    lib.ss_filter_submaze.argtypes = [P, P, P, ctypes.c_int, I32, I32, I32,
                                      I32, I64, P, P, P]
    lib.ss_gather_pairs.argtypes = [P, P, P, I32, P, P, I64, P, P, P]
    lib.ss_server_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, SZ,
                                     ctypes.c_int]
    lib.ss_server_submit.argtypes = [P, P, P, P, P, I64,
                                     ctypes.POINTER(ctypes.c_uint64)]
    lib.ss_server_poll.argtypes = [P, ctypes.c_uint64]
    lib.ss_server_wait.argtypes = [P, ctypes.c_uint64, I64]
    lib.ss_server_fetch.argtypes = [P, ctypes.c_uint64, P, P,
                                    ctypes.POINTER(ctypes.c_double)]
    lib.ss_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
    lib.ss_server_reset_stats.argtypes = [P]
    lib.ss_server_destroy.argtypes = [P]
    lib.ss_set_tuning.argtypes = [P, ctypes.c_int, ctypes.c_int]
    lib.ss_get_tuning.argtypes = [P, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]
    lib.ss_autotune.argtypes = [P, P, P, P, P, I32, P, I32, I64, P, P, P,
                                ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
    for name in EXPORTED:
        getattr(lib, name)  # raises AttributeError if a symbol is missing
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().ss_strerror(int(code)).decode()


def _check(rc: int, what: str):
    if rc != SS_OK:
        raise SSError(rc, what)


# ---- same-name functions (pointers as ints; 0 = NULL) --------------------

def ss_create(device: int = 0, workspace_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().ss_create(ctypes.byref(h), device, workspace_bytes),
           "ss_create")
    return h.value


def ss_destroy(ctx: int) -> None:
    _check(load().ss_destroy(ctx), "ss_destroy")


def ss_version() -> int:
    return load().ss_version()


def ss_packed_words(m: int) -> int:
    return int(load().ss_packed_words(m))


def ss_sliced_words(m: int, n: int) -> int:
    return int(load().ss_sliced_words(m, n))


def ss_pack_sliced(ctx, ascii, m, n, sliced, stream) -> int:
    return load().ss_pack_sliced(ctx, ascii or None, m, n, sliced or None,
                                 stream or None)


def ss_filter_sweep(ctx, reads, refs, fmt, m, e_list, n_e, n, stream,
                    out_accept, out_obstacles) -> int:
    return load().ss_filter_sweep(ctx, reads or None, refs or None, fmt, m,
                                  e_list or None, n_e, n, stream or None,
                                  out_accept or None, out_obstacles or None)


def ss_filter_segments(ctx, segs, n_seg, fmt, flags, stream) -> int:
    """segs: a ctypes array of Segment (or None with n_seg 0)."""
    return load().ss_filter_segments(ctx, segs, n_seg, fmt, flags,
                                     stream or None)


def ss_pack(ctx, ascii, offsets, lengths, m, n, packed, packed_offsets,
            stream) -> int:
    return load().ss_pack(ctx, ascii or None, offsets or None,
                          lengths or None, m, n, packed or None,
                          packed_offsets or None, stream or None)


def ss_filter_batch(ctx, reads, refs, fmt, offsets, lengths, m, E, e, n,
                    flags, stream, out_accept, out_obstacles) -> int:
    return load().ss_filter_batch(ctx, reads or None, refs or None, fmt,
                                  offsets or None, lengths or None, m,
                                  E or None, e, n, flags, stream or None,
                                  out_accept or None, out_obstacles or None)


def ss_filter_host(ctx, reads, refs, fmt, m, e_list, n_e, n, out_accept,
                   out_obstacles) -> int:
    return load().ss_filter_host(ctx, reads or None, refs or None, fmt, m,
                                 e_list or None, n_e, n, out_accept or None,
                                 out_obstacles or None)


def ss_sync(ctx, stream=0) -> int:
    return load().ss_sync(ctx, stream or None)


def ss_get_counters(ctx) -> Counters:
    c = Counters()
    _check(load().ss_get_counters(ctx, ctypes.byref(c)), "ss_get_counters")
    return c


def ss_filter_batch_noalloc(reads, refs, offsets, lengths, m, E, e, n,
                            stream, out_accept, out_obstacles) -> int:
    """Allocation-free bucketed filter (packed input, current device)."""
    return load().ss_filter_batch_noalloc(
        reads or None, refs or None, offsets or None, lengths or None, m,
        E or None, e, n, stream or None, out_accept or None,
        out_obstacles or None)


def ss_set_tuning(ctx, rw_max_e: int, cw_subgrid: int) -> int:
    return load().ss_set_tuning(ctx, rw_max_e, cw_subgrid)


def ss_get_tuning(ctx):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().ss_get_tuning(ctx, ctypes.byref(a), ctypes.byref(b)),
           "ss_get_tuning")
    return a.value, b.value


def ss_autotune(ctx, reads, refs, offsets, lengths, m, E, e, n, stream,
                out_accept, out_obstacles, reps=3):
    best = ctypes.c_float()
    rc = load().ss_autotune(ctx, reads or None, refs or None, offsets or None,
                            lengths or None, m, E or None, e, n,
                            stream or None, out_accept or None,
                            out_obstacles or None, reps, ctypes.byref(best))
    _check(rc, "ss_autotune")
    return best.value


# ---- torch marshalling ------------------------------------------------------

def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _dptr(t, device: int, what: str, nbytes: int = 0) -> int:
    """Address of a contiguous CUDA tensor on `device` holding at least
    `nbytes` (0 for None).  The C ABI takes plain device pointers and cannot
    check them: a host tensor, another device's tensor or a short buffer
    would be read or written out of bounds by the kernels."""
    if t is None:
        return 0
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what}: expected a CUDA tensor on cuda:{device}")
    if t.device.index != device:
        raise ValueError(f"{what}: tensor on cuda:{t.device.index}, "
                         f"context on cuda:{device}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    have = t.numel() * t.element_size()
    if have < nbytes:
        raise ValueError(f"{what}: {have} bytes, the call needs {nbytes}")
    return int(t.data_ptr())


def _hptr(t, what: str, nbytes: int = 0) -> int:
    """Address of a contiguous host tensor holding at least `nbytes`."""
    if getattr(t, "is_cuda", False):
        raise ValueError(f"{what}: expected a host (CPU) tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    have = t.numel() * t.element_size()
    if have < nbytes:
        raise ValueError(f"{what}: {have} bytes, the call needs {nbytes}")
    return int(t.data_ptr())


def _seq_bytes(fmt: int, n: int, m: int) -> int:
    """Bytes of n fixed-stride sequences of m bases in format fmt."""
    if n <= 0 or m <= 0:
        return 0
    if fmt == SS_FMT_SLICED2:
        return 4 * ss_sliced_words(m, n)
    return n * m if fmt == SS_FMT_ASCII else n * 4 * ss_packed_words(m)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Filter:
    """A context bound to one CUDA device; methods take torch tensors."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0):
        self.device = device
        self.ctx = ss_create(device, workspace_bytes)

    def close(self):
        if self.ctx:
            ss_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, ascii, m: int = 0, n: Optional[int] = None, offsets=None,
             lengths=None, out=None, out_offsets=None, stream=None):
        """ASCII (uint8, device) -> packed int32 words (device)."""
        import torch
        if offsets is None:
            n = ascii.shape[0] if n is None else n
            if out is None:
                out = torch.empty(n * ss_packed_words(m), dtype=torch.int32,
                                  device=ascii.device)
        else:
            n = lengths.shape[0]
        d = self.device
        fixed = offsets is None
        rc = ss_pack(self.ctx,
                     _dptr(ascii, d, "ascii",
                           _seq_bytes(SS_FMT_ASCII, n, m) if fixed else 0),
                     _dptr(offsets, d, "offsets", 8 * n),
                     _dptr(lengths, d, "lengths", 4 * n), m, n,
                     _dptr(out, d, "out",
                           _seq_bytes(SS_FMT_PACKED2, n, m) if fixed else 0),
                     _dptr(out_offsets, d, "out_offsets", 8 * n),
                     _stream_handle(stream))
        _check(rc, "ss_pack")
        return out

    def pack_sliced(self, ascii, m: int, n: Optional[int] = None, out=None,
                    stream=None):
        """Fixed-stride ASCII (uint8, device) -> the bit-sliced layout
        (int32 words, device, ss_sliced_words(m, n) of them)."""
        import torch
        n = ascii.shape[0] if n is None else n
        if out is None:
            out = torch.empty(max(ss_sliced_words(m, n), 1),
                              dtype=torch.int32, device=ascii.device)
        d = self.device
        rc = ss_pack_sliced(self.ctx,
                            _dptr(ascii, d, "ascii",
                                  _seq_bytes(SS_FMT_ASCII, n, m)), m, n,
                            _dptr(out, d, "out",
                                  _seq_bytes(SS_FMT_SLICED2, n, m)),
                            _stream_handle(stream))
        _check(rc, "ss_pack_sliced")
        return out

    def filter(self, reads, refs, *, m: int = 0, e: int = 0, n=None,
               fmt: int = SS_FMT_PACKED2, offsets=None, lengths=None, E=None,
               flags: int = SS_MODE_AUTO, out_accept=None,
               out_obstacles=None, stream=None, sync: bool = False):
        """Filter device pairs; returns (accept uint8, obstacles int32)."""
        import torch
        if n is None:
            n = lengths.shape[0] if lengths is not None else reads.shape[0]
        dev = reads.device
        if out_accept is None:
            out_accept = torch.empty(n, dtype=torch.uint8, device=dev)
        if out_obstacles is None:
            out_obstacles = torch.empty(n, dtype=torch.int32, device=dev)
        d = self.device
        seq = _seq_bytes(fmt, n, m) if offsets is None else 0
        rc = ss_filter_batch(self.ctx, _dptr(reads, d, "reads", seq),
                             _dptr(refs, d, "refs", seq), fmt,
                             _dptr(offsets, d, "offsets", 8 * n),
                             _dptr(lengths, d, "lengths", 4 * n), m,
                             _dptr(E, d, "E", 4 * n), e, n, flags,
                             _stream_handle(stream),
                             _dptr(out_accept, d, "out_accept", n),
                             _dptr(out_obstacles, d, "out_obstacles", 4 * n))
        _check(rc, "ss_filter_batch")
        if sync:
            self.sync(stream)
        return out_accept, out_obstacles

    def filter_sweep(self, reads, refs, *, m: int, e, n: int,
                     fmt: int = SS_FMT_SLICED2, out_accept=None,
                     out_obstacles=None, stream=None, sync: bool = False):
        """Device pairs filtered at every threshold of the list e; outputs
        (accept uint8, obstacles int32) of shape (len(e), n), device."""
        import torch
        es = [int(x) for x in e]
        e_arr = (ctypes.c_int32 * len(es))(*es)
        k = len(es)
        dev = reads.device
        if out_accept is None:
            out_accept = torch.empty((k, n), dtype=torch.uint8, device=dev)
        if out_obstacles is None:
            out_obstacles = torch.empty((k, n), dtype=torch.int32,
                                        device=dev)
        d = self.device
        seq = _seq_bytes(fmt, n, m)
        rc = ss_filter_sweep(self.ctx, _dptr(reads, d, "reads", seq),
                             _dptr(refs, d, "refs", seq), fmt, m,
                             ctypes.addressof(e_arr), k, n,
                             _stream_handle(stream),
                             _dptr(out_accept, d, "out_accept", k * n),
                             _dptr(out_obstacles, d, "out_obstacles",
                                   4 * k * n))
        _check(rc, "ss_filter_sweep")
        if sync:
            self.sync(stream)
        return out_accept, out_obstacles

    def filter_segments(self, segments, *, fmt: int = SS_FMT_SLICED2,
                        graph: bool = True, stream=None, sync: bool = False):
        """Uniform batches filtered by one call (ss_filter_segments).
        ``segments``: (reads, refs, m, e, n) tuples of device tensors in the
        format ``fmt``, m the length of reads and references or a pair
        (read length, reference length); returns one (accept uint8[n],
        obstacles int32[n]) pair of new device tensors per segment, in the
        given order.  A 6-tuple (reads, refs, m, e, n, (out_accept,
        out_obstacles)) writes to the given tensors instead."""
        import torch
        d = self.device
        arr = (Segment * max(len(segments), 1))()
        outs = []
        for i, sg in enumerate(segments):
            reads, refs, m, e, n = sg[:5]
            m, m_ref = (m, m) if isinstance(m, int) else m
            m, m_ref, e, n = int(m), int(m_ref), int(e), int(n)
            if len(sg) > 5:
                acc, obs = sg[5]
            else:
                acc = torch.empty(n, dtype=torch.uint8, device=reads.device)
                obs = torch.empty(n, dtype=torch.int32, device=reads.device)
            arr[i] = Segment(
                _dptr(reads, d, "reads", _seq_bytes(fmt, n, m)) or None,
                _dptr(refs, d, "refs", _seq_bytes(fmt, n, m_ref)) or None,
                n, m, e, _dptr(acc, d, "out_accept", n) or None,
                _dptr(obs, d, "out_obstacles", 4 * n) or None, m_ref)
            outs.append((acc, obs))
        rc = ss_filter_segments(self.ctx, arr if segments else None,
                                len(segments), fmt,
                                0 if graph else SS_FLAG_NO_GRAPH,
                                _stream_handle(stream))
        _check(rc, "ss_filter_segments")
        if sync:
            self.sync(stream)
        return outs

    def filter_host(self, reads, refs, *, m: int, e, n=None,
                    fmt: int = SS_FMT_ASCII, out_accept=None,
                    out_obstacles=None):
        """Host (CPU, ideally pinned) tensors in and out.  ``e`` is one
        threshold or a list; outputs have shape (len(e), n) for a list."""
        import torch
        n = reads.shape[0] if n is None else n
        es = [int(e)] if isinstance(e, int) else [int(x) for x in e]
        e_arr = (ctypes.c_int32 * len(es))(*es)
        if out_accept is None:
            out_accept = torch.empty((len(es), n), dtype=torch.uint8,
                                     pin_memory=True)
        if out_obstacles is None:
            out_obstacles = torch.empty((len(es), n), dtype=torch.int32,
                                        pin_memory=True)
        seq = _seq_bytes(fmt, n, m)
        k = len(es)
        rc = ss_filter_host(self.ctx, _hptr(reads, "reads", seq),
                            _hptr(refs, "refs", seq), fmt, m,
                            ctypes.addressof(e_arr), k, n,
                            _hptr(out_accept, "out_accept", k * n),
                            _hptr(out_obstacles, "out_obstacles", 4 * k * n))
        _check(rc, "ss_filter_host")
        if isinstance(e, int):
            return out_accept[0], out_obstacles[0]
        return out_accept, out_obstacles

    def autotune(self, reads, refs, *, m: int = 0, e: int = 0, n=None,
                 offsets=None, lengths=None, E=None, reps: int = 3,
                 out_accept=None, out_obstacles=None, stream=None):
        """Time every tuning of the bucketed form on this (packed) batch and
        keep the fastest; returns (rw_max_e, cw_subgrid, best ms)."""
        import torch
        if n is None:
            n = lengths.shape[0] if lengths is not None else reads.shape[0]
        if out_accept is None:
            out_accept = torch.empty(n, dtype=torch.uint8, device=reads.device)
        if out_obstacles is None:
            out_obstacles = torch.empty(n, dtype=torch.int32,
                                        device=reads.device)
        d = self.device
        seq = _seq_bytes(SS_FMT_PACKED2, n, m) if offsets is None else 0
        ms = ss_autotune(self.ctx, _dptr(reads, d, "reads", seq),
                         _dptr(refs, d, "refs", seq),
                         _dptr(offsets, d, "offsets", 8 * n),
                         _dptr(lengths, d, "lengths", 4 * n), m,
                         _dptr(E, d, "E", 4 * n), e, n,
                         _stream_handle(stream),
                         _dptr(out_accept, d, "out_accept", n),
                         _dptr(out_obstacles, d, "out_obstacles", 4 * n),
                         reps)
        rmax, k = ss_get_tuning(self.ctx)
        return rmax, k, ms

    def set_tuning(self, rw_max_e: int, cw_subgrid: int):
        _check(ss_set_tuning(self.ctx, rw_max_e, cw_subgrid), "ss_set_tuning")

    def edit_distance(self, reads, refs, *, m: int, e: int, n=None,
                      out=None, stream=None):
        """min(ED, e+1) of fixed-stride packed pairs (device int32[n])."""
        import torch
        n = reads.shape[0] if n is None else n
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=reads.device)
        d = self.device
        seq = _seq_bytes(SS_FMT_PACKED2, n, m)
        rc = load().ss_edit_distance_banded(
            self.ctx, _dptr(reads, d, "reads", seq) or None,
            _dptr(refs, d, "refs", seq) or None, SS_FMT_PACKED2, m, e, n,
            _stream_handle(stream) or None,
            _dptr(out, d, "out", 4 * n) or None)
        _check(rc, "ss_edit_distance_banded")
        return out

    def filter_submaze(self, reads, refs, *, m: int, e: int, t: int, y: int,
                       n=None, fmt: int = SS_FMT_PACKED2, stream=None):
        """Sub-maze approximate mode (Section 2.5) on fixed-stride packed
        (pair-major or bit-sliced) pairs; returns (accept, obstacles)."""
        import torch
        n = reads.shape[0] if n is None else n
        acc = torch.empty(max(n, 1), dtype=torch.uint8, device=reads.device)
        obs = torch.empty(max(n, 1), dtype=torch.int32, device=reads.device)
        d = self.device
        seq = _seq_bytes(fmt, n, m)
        rc = load().ss_filter_submaze(self.ctx, _dptr(reads, d, "reads", seq),
                                      _dptr(refs, d, "refs", seq),
                                      fmt, m, e, t, y, n,
                                      _stream_handle(stream) or None,
                                      _ptr(acc), _ptr(obs))
        _check(rc, "ss_filter_submaze")
        return acc[:n], obs[:n]

    def filter_unequal(self, reads, read_off, read_len, refs, ref_off,
                       ref_len, *, e: int = 0, E=None, stream=None):
        """Pairs of possibly different lengths (packed, device arrays of
        word offsets and base lengths); returns (accept, obstacles)."""
        import torch
        n = read_len.shape[0]
        dev = read_len.device
        acc = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
        obs = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        d = self.device
        rc = load().ss_filter_unequal(
            self.ctx, _dptr(reads, d, "reads"),
            _dptr(read_off, d, "read_off", 8 * n),
            _dptr(read_len, d, "read_len", 4 * n), _dptr(refs, d, "refs"),
            _dptr(ref_off, d, "ref_off", 8 * n),
            _dptr(ref_len, d, "ref_len", 4 * n), _dptr(E, d, "E", 4 * n), e,
            n, _stream_handle(stream) or None, _ptr(acc), _ptr(obs))
        _check(rc, "ss_filter_unequal")
        return acc[:n], obs[:n]

    def check_wait_timeout(self, limit_ns: int, stream=None):
        """Launch the bounded-wait self-test; the next sync raises
        SSError(SS_ERR_TIMEOUT)."""
        rc = load().ss_check_wait_timeout(self.ctx, int(limit_ns),
                                          _stream_handle(stream) or None)
        _check(rc, "ss_check_wait_timeout")

    def compact(self, accept, stream=None):
        """Indices of accepted pairs, in order: (device int64[n] buffer,
        device int64 count)."""
        import torch
        n = accept.shape[0]
        idx = torch.empty(max(n, 1), dtype=torch.int64, device=accept.device)
        cnt = torch.empty(1, dtype=torch.int64, device=accept.device)
        rc = load().ss_compact_accepted(self.ctx,
                                        _dptr(accept, self.device, "accept")
                                        or None, n,
                                        _stream_handle(stream) or None,
                                        _ptr(idx), _ptr(cnt))
        _check(rc, "ss_compact_accepted")
        return idx, cnt

    def gather(self, reads, refs, index, count, *, m: int, n: int,
               stream=None):
        """Dense packed copies of the pairs listed in index[:count] (n slots
        of ceil(m/16) words each)."""
        import torch
        w16 = ss_packed_words(m)
        out_q = torch.zeros(max(n * w16, 1), dtype=torch.int32,
                            device=reads.device)
        out_r = torch.zeros_like(out_q)
        d = self.device
        rc = load().ss_gather_pairs(self.ctx, _dptr(reads, d, "reads"),
                                    _dptr(refs, d, "refs"), m,
                                    _dptr(index, d, "index"),
                                    _dptr(count, d, "count", 8), n,
                                    _stream_handle(stream) or None,
                                    _ptr(out_q), _ptr(out_r))
        _check(rc, "ss_gather_pairs")
        return out_q, out_r

    def edit_distance_varlen(self, reads, refs, offsets, lengths, E,
                             stream=None):
        """min(ED, E[p]+1) of packed pairs with per-pair word offsets,
        lengths and thresholds (E <= 511); device int32[n]."""
        import torch
        n = lengths.shape[0]
        out = torch.empty(max(n, 1), dtype=torch.int32, device=lengths.device)
        d = self.device
        rc = load().ss_edit_distance_varlen(
            self.ctx, _dptr(reads, d, "reads"), _dptr(refs, d, "refs"),
            _dptr(offsets, d, "offsets", 8 * n),
            _dptr(lengths, d, "lengths", 4 * n), _dptr(E, d, "E", 4 * n), n,
            _stream_handle(stream) or None, _ptr(out))
        _check(rc, "ss_edit_distance_varlen")
        return out[:n]

    def confusion(self, accept, ed, *, e: int, stream=None):
        """(true accepts, false accepts, false rejects, true rejects)."""
        import torch
        counts = torch.zeros(4, dtype=torch.int64, device=accept.device)
        n = accept.shape[0]
        d = self.device
        rc = load().ss_filter_confusion(
            self.ctx, _dptr(accept, d, "accept", n), _dptr(ed, d, "ed", 4 * n),
            n, e, _stream_handle(stream) or None, _ptr(counts))
        _check(rc, "ss_filter_confusion")
        return tuple(int(x) for x in counts.cpu().tolist())

    def sync(self, stream=None):
        """Wait for the stream (default: torch's current stream) and raise
        any error the kernels latched."""
        _check(ss_sync(self.ctx, _stream_handle(stream)), "ss_sync")

    def counters(self) -> Counters:
        return ss_get_counters(self.ctx)


class Server:
    """Continuous-batching request server (ss_server_* of include/ss.h).

    Requests are numpy arrays in host memory: concatenated ASCII reads and
    refs, per-pair int32 lengths and thresholds.  The arrays are kept alive
    here until the request is fetched, as the C API requires."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0,
                 slots: int = 3):
        h = ctypes.c_void_p()
        _check(load().ss_server_create(ctypes.byref(h), device,
                                       hbm_budget_bytes, slots),
               "ss_server_create")
        self.h = h.value
        self._keep = {}

    def close(self):
        if self.h:
            load().ss_server_destroy(self.h)
            self.h = 0
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, reads, refs, lengths, E) -> int:
        import numpy as np
        reads = np.ascontiguousarray(reads, dtype=np.uint8)
        refs = np.ascontiguousarray(refs, dtype=np.uint8)
        lengths = np.ascontiguousarray(lengths, dtype=np.int32)
        E = np.ascontiguousarray(E, dtype=np.int32)
        # the library copies sum(lengths) bytes of each from host memory
        need = int(np.clip(lengths, 0, None).sum(dtype=np.int64))
        if reads.size < need or refs.size < need:
            raise ValueError(f"reads/refs hold {reads.size}/{refs.size} "
                             f"bytes, the lengths need {need}")
        if E.size < lengths.size:
            raise ValueError(f"{E.size} thresholds for {lengths.size} pairs")
        t = ctypes.c_uint64()
        rc = load().ss_server_submit(
            self.h, reads.ctypes.data if reads.size else None,
            refs.ctypes.data if refs.size else None, lengths.ctypes.data,
            E.ctypes.data, len(lengths), ctypes.byref(t))
        _check(rc, "ss_server_submit")
        self._keep[t.value] = (reads, refs, lengths, E)
        return t.value

    def poll(self, ticket: int) -> int:
        return load().ss_server_poll(self.h, ticket)

    def wait(self, ticket: int, timeout_s: float = 600.0) -> int:
        return load().ss_server_wait(self.h, ticket, int(timeout_s * 1e6))

    def fetch(self, ticket: int):
        """(status, accept uint8[n], obstacles int32[n], latency seconds)."""
        import numpy as np
        n = len(self._keep[ticket][2])
        acc = np.empty(max(n, 1), np.uint8)
        obs = np.empty(max(n, 1), np.int32)
        lat = ctypes.c_double()
        rc = load().ss_server_fetch(self.h, ticket, acc.ctypes.data,
                                    obs.ctypes.data, ctypes.byref(lat))
        if rc != SS_ERR_BUSY:
            self._keep.pop(ticket, None)
        return rc, acc[:n], obs[:n], lat.value

    def stats(self) -> dict:
        st = ServerStats()
        rc = load().ss_server_get_stats(self.h, ctypes.byref(st))
        d = st.as_dict()
        d["status"] = rc
        return d

    def reset_stats(self):
        load().ss_server_reset_stats(self.h)
