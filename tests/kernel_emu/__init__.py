"""Host build of the library's routing functions (test harness only)."""
import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_1910_09020_gb300", "csrc")
SRC = os.path.join(HERE, "emu.cu")
OUT = os.path.join(HERE, "_build", "libemu.so")
_lib = None


def _deps():
    return [SRC] + [os.path.join(CSRC, f) for f in os.listdir(CSRC)
                    if f.endswith((".cuh", ".h"))]


def load():
    global _lib
    if _lib is not None:
        return _lib
    stale = (not os.path.exists(OUT) or
             any(os.path.getmtime(d) > os.path.getmtime(OUT) for d in _deps()))
    if stale:
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        tmp = OUT + f".tmp{os.getpid()}"
        nvcc = os.environ.get("NVCC", "nvcc")
        if not os.path.exists(nvcc) and os.path.exists("/usr/local/cuda/bin/nvcc"):
            nvcc = "/usr/local/cuda/bin/nvcc"
        subprocess.check_call([
            nvcc, "-std=c++17", "-O2", "-gencode",
            "arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC",
            "-shared", "-I", CSRC, SRC, "-o", tmp])
        os.replace(tmp, OUT)
    lib = ctypes.CDLL(OUT)
    P = ctypes.c_void_p
    lib.emu_rw_exact.argtypes = [P, P, ctypes.c_int, ctypes.c_int]
    lib.emu_rw_cols.argtypes = [P, P, ctypes.c_int, ctypes.c_int]
    lib.emu_rw_staged.argtypes = [P, P] + [ctypes.c_int] * 3
    lib.emu_rw_runtime.argtypes = [P, P, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int]
    lib.emu_cw.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.emu_class_of.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.emu_ed.argtypes = [P, P, ctypes.c_int, ctypes.c_int]
    lib.emu_pack_chunk.argtypes = [P, P]
    lib.emu_pack_chunk.restype = ctypes.c_uint32
    lib.emu_pack_chunk_pairs.argtypes = [P, P]
    lib.emu_pack_chunk_pairs.restype = ctypes.c_uint32
    lib.emu_pack_window.argtypes = [ctypes.c_uint32] * 3
    lib.emu_pack_window.restype = ctypes.c_uint32
    lib.emu_unequal.argtypes = [P, ctypes.c_int, P, ctypes.c_int,
                                ctypes.c_int]
    lib.emu_unequal_form.argtypes = [P, ctypes.c_int, P, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int]
    lib.emu_unequal_staged.argtypes = [P, ctypes.c_int, P, ctypes.c_int,
                                       ctypes.c_int]
    lib.emu_unequal_exact.argtypes = [P, ctypes.c_int, P, ctypes.c_int,
                                      ctypes.c_int]
    lib.emu_submaze.argtypes = [P, P, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int]
    lib.emu_submaze_rows.argtypes = [P, P, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int]
    lib.emu_submaze_cols.argtypes = [P, P, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int]
    lib.emu_submaze_staged.argtypes = [P, P] + [ctypes.c_int] * 5
    lib.emu_sliced.argtypes = [P, P, ctypes.c_int64, ctypes.c_int,
                               ctypes.c_int, P, P]
    lib.emu_transpose32.argtypes = [P, P]
    lib.emu_sliced_submaze.argtypes = [P, P, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, P, P]
    lib.emu_sliced_set.argtypes = [P, P, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_int, P, P]
    lib.emu_sliced_free.argtypes = [P, P, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, P, P]
    _lib = lib
    return lib
