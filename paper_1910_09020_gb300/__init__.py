"""SneakySnake pre-alignment filter for GB300 (sm_103a).

The filter itself lives in the CUDA library ``csrc/`` behind the C ABI
declared in ``include/ss.h``; :mod:`paper_1910_09020_gb300.binding` is the
thin ctypes layer over it and :mod:`paper_1910_09020_gb300.synth` the seeded
workload generator.  Importing this package loads nothing; the binding loads
the shared library on first use and raises if it is missing.
"""

__all__ = ["binding", "synth", "build"]
