"""Measured integer-pipe peaks of the GPU (denominator of the filter's ALU
roofline).  Built by paper_1910_09020_gb300.build into _build/libss_peaks.so.
"""
from __future__ import annotations

import ctypes

from .. import build as _build

KINDS = {"lop3": 0, "add": 1, "shf": 2, "bfind": 3}


def measure(device: int = 0) -> dict:
    """Lane-operations per second of each instruction kind."""
    lib = ctypes.CDLL(_build.build_peaks())
    lib.ss_peak_int.argtypes = [ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double)]
    out = {}
    for name, k in KINDS.items():
        r, ms = ctypes.c_double(), ctypes.c_double()
        rc = lib.ss_peak_int(device, k, ctypes.byref(r), ctypes.byref(ms))
        if rc != 0:
            raise RuntimeError(f"peak microbenchmark {name} failed: {rc}")
        out[name] = r.value
    return out
