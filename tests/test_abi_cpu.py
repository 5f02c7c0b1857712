"""The C-ABI library builds, loads and exports every symbol include/ss.h
declares; host-only argument checks (no kernel launches, no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1910_09020_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(ss_\w+)\s*\(", text,
                            flags=re.M)
    return sorted(set(names))


def test_library_builds_and_loads():
    path = build.build()
    assert os.path.exists(path)
    lib = binding.load()
    assert isinstance(lib, ctypes.CDLL)


def test_every_declared_symbol_is_exported():
    lib = binding.load()
    decl = declared_functions()
    assert len(decl) >= 10
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == sorted(
        n for n in decl if n in binding.EXPORTED)
    assert set(decl) <= set(binding.EXPORTED), set(decl) - set(binding.EXPORTED)


def test_host_only_functions():
    assert binding.ss_version() >= 100
    assert binding.ss_packed_words(0) == 0
    assert binding.ss_packed_words(1) == 1
    assert binding.ss_packed_words(16) == 1
    assert binding.ss_packed_words(17) == 2
    assert binding.ss_packed_words(100000) == 6250
    assert "A/C/G/T" in binding.strerror(binding.SS_ERR_INVALID_BASE)
    assert binding.strerror(12345) == "unknown status"


def test_null_context_rejected():
    lib = binding.load()
    assert binding.ss_filter_batch(0, 1, 1, 0, 0, 0, 10, 0, 1, 5, 0, 0, 1,
                                   1) == binding.SS_ERR_INVALID_ARG
    assert binding.ss_sync(0) == binding.SS_ERR_INVALID_ARG
    assert binding.ss_filter_segments(0, None, 0, binding.SS_FMT_SLICED2, 0,
                                      0) == binding.SS_ERR_INVALID_ARG
    assert lib.ss_destroy(None) == binding.SS_OK


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = binding.load().ss_create(ctypes.byref(h), 0, 0)
    assert rc in (binding.SS_ERR_CUDA, binding.SS_ERR_INVALID_ARG)
    assert not h.value


def test_submaze_rejects_bad_arguments_without_gpu():
    lib = binding.load()
    P = ctypes.c_void_p
    for args in [(None, P(1), P(1), binding.SS_FMT_PACKED2, 100, 3, 8, 3, 1),
                 ]:
        rc = lib.ss_filter_submaze(*args, None, P(1), P(1))
        assert rc == binding.SS_ERR_INVALID_ARG


def test_wait_self_test_rejects_null_context():
    lib = binding.load()
    assert lib.ss_check_wait_timeout(None, 50_000_000, None) == \
        binding.SS_ERR_INVALID_ARG


def test_binding_rejects_host_short_or_strided_buffers():
    """The C ABI takes plain pointers and cannot check them, so the binding
    refuses what the kernels would read or write out of bounds: a host
    tensor where a device one is due (and the reverse), a strided view, or
    fewer bytes than the call's shape needs."""
    torch = pytest.importorskip("torch")
    h = torch.zeros(64, dtype=torch.uint8)
    with pytest.raises(ValueError, match="CUDA tensor"):
        binding._dptr(h, 0, "reads")
    assert binding._dptr(None, 0, "E") == 0
    assert binding._hptr(h, "reads", 64) == h.data_ptr()
    with pytest.raises(ValueError, match="needs 65"):
        binding._hptr(h, "reads", 65)
    with pytest.raises(ValueError, match="contiguous"):
        binding._hptr(h.view(8, 8).t(), "reads")
    assert binding._seq_bytes(binding.SS_FMT_ASCII, 3, 100) == 300
    assert binding._seq_bytes(binding.SS_FMT_PACKED2, 3, 100) == 3 * 7 * 4
    assert binding._seq_bytes(binding.SS_FMT_PACKED2, 0, 100) == 0
    assert binding._seq_bytes(binding.SS_FMT_ASCII, 5, 0) == 0


def test_server_submit_checks_request_sizes():
    """A request's reads and refs must hold sum(lengths) bytes each (the
    library copies that much from host memory) and one threshold per pair;
    checked before the library is called (no server needed)."""
    np = pytest.importorskip("numpy")
    S = object.__new__(binding.Server)  # no device: the checks come first
    S.h, S._keep = 0, {}
    with pytest.raises(ValueError, match="need 200"):
        S.submit(np.zeros(100, np.uint8), np.zeros(200, np.uint8),
                 [100, 100], [1, 1])
    with pytest.raises(ValueError, match="thresholds"):
        S.submit(np.zeros(200, np.uint8), np.zeros(200, np.uint8),
                 [100, 100], [1])
