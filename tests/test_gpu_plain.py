"""GPU parity of the pack kernel and the plain (uniform m, E) filter against
the CPU oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import oracle
from gpu_util import (FMT_ASCII, FMT_PACKED2, assert_same, gpu_filter_fixed,
                      oracle_fixed, recipes, to_dev, torch_cuda)
from paper_1910_09020_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    torch_cuda()
    f = binding.Filter(0)
    yield f
    f.close()


# ---- K1 pack ------------------------------------------------------------------

@pytest.mark.parametrize("m", [1, 15, 16, 17, 31, 33, 100, 150, 250, 1000])
def test_pack_matches_reference_packer(F, m):
    reads, _ = synth.pairs_fixed(101, 0, 300, m, synth.SHORT_UNIFORM_K)
    rng = np.random.default_rng(m)
    lower = rng.random(reads.shape) < 0.3
    reads = np.where(lower, reads | 0x20, reads).astype(np.uint8)
    packed = F.pack(to_dev(reads.reshape(-1)), m=m, n=300)
    F.sync()
    got = packed.cpu().numpy().view(np.uint32).reshape(300, -1)
    for p in range(300):
        want = oracle.pack_reference(reads[p].tobytes())
        assert (got[p] == want).all(), p


def test_pack_varlen_matches_reference_packer(F):
    torch = torch_cuda()
    L = synth.log_uniform(5, 0, 200, 1, 3000)
    reads, _, off = synth.pairs_varlen(5, 0, L, synth.rate_recipe(0.1))
    words = (L.astype(np.int64) + 15) // 16
    poff = np.zeros(len(L) + 1, np.int64)
    np.cumsum(words, out=poff[1:])
    out = torch.zeros(int(poff[-1]) + 1, dtype=torch.int32, device="cuda")
    F.pack(to_dev(reads), offsets=to_dev(off), lengths=to_dev(L), out=out,
           out_offsets=to_dev(poff))
    F.sync()
    got = out.cpu().numpy().view(np.uint32)
    for p in range(len(L)):
        seq = reads[off[p]:off[p] + L[p]].tobytes()
        want = oracle.pack_reference(seq)
        assert (got[poff[p]:poff[p + 1]] == want).all(), p


@pytest.mark.parametrize("m,shift", [(37, 0), (100, 0), (128, 0),
                                     (100, 1), (100, 4), (23, 3)])
def test_pack_many_ctas_and_unaligned_input(F, m, shift):
    """Enough pairs for hundreds of CTAs (each staging its own span of the
    byte stream), with the input both 16-byte aligned and not."""
    torch = torch_cuda()
    n = 40000
    reads, _ = synth.pairs_fixed(202 + m, 0, n, m, synth.SHORT_POISSON)
    rng = np.random.default_rng(m + shift)
    lower = rng.random(reads.shape) < 0.5
    reads = np.where(lower, reads | 0x20, reads).astype(np.uint8)
    buf = torch.zeros(n * m + 64, dtype=torch.uint8, device="cuda")
    buf[shift:shift + n * m] = to_dev(reads.reshape(-1))
    packed = F.pack(buf[shift:shift + n * m], m=m, n=n)
    F.sync()
    got = packed.cpu().numpy().view(np.uint32).reshape(n, -1)
    for p in range(n):
        want = oracle.pack_reference(reads[p].tobytes())
        assert (got[p] == want).all(), p


@pytest.mark.parametrize("where", ["first", "cta_edge", "last"])
def test_pack_invalid_base_anywhere_latches(F, where):
    n, m = 40000, 100
    reads, _ = synth.pairs_fixed(9, 0, n, m, synth.SHORT_UNIFORM_K)
    flat = reads.reshape(-1).copy()
    pos = {"first": 0, "cta_edge": 1024 * 16 - 1, "last": n * m - 1}[where]
    flat[pos] = ord("u")
    F.pack(to_dev(flat), m=m, n=n)
    with pytest.raises(binding.SSError) as ei:
        F.sync()
    assert ei.value.code == binding.SS_ERR_INVALID_BASE
    F.sync()


def test_pack_invalid_base_latches(F):
    reads, _ = synth.pairs_fixed(3, 0, 64, 100, synth.SHORT_UNIFORM_K)
    reads[17, 55] = ord("N")
    F.pack(to_dev(reads.reshape(-1)), m=100, n=64)
    with pytest.raises(binding.SSError) as ei:
        F.sync()
    assert ei.value.code == binding.SS_ERR_INVALID_BASE
    F.sync()  # cleared


# ---- plain filter -----------------------------------------------------------------

def test_worked_example(F):
    """Fig. 2: R = GGTGCAGAGCTC, Q = GGTGAGAGTTGT, E = 3 -> 3 obstacles,
    accept."""
    Q = np.frombuffer(b"GGTGAGAGTTGT", np.uint8).reshape(1, 12)
    R = np.frombuffer(b"GGTGCAGAGCTC", np.uint8).reshape(1, 12)
    for fmt in (FMT_ASCII, FMT_PACKED2):
        acc, obs = gpu_filter_fixed(F, Q, R, 3, fmt)
        assert (acc[0], obs[0]) == (1, 3)


def test_config1_all_pairs(F):
    """10,000 pairs of 100 bp, k ~ U{0..10} edits, ASCII input, E = 5."""
    reads, refs = synth.pairs_fixed(1910_09020 + 1, 0, 10000, 100,
                                    synth.SHORT_UNIFORM_K)
    acc, obs = gpu_filter_fixed(F, reads, refs, 5, FMT_ASCII)
    oacc, oobs = oracle_fixed(reads, refs, 5)
    assert_same(acc, obs, oacc, oobs, "config 1")
    assert 0 < oacc.mean() < 1


SIZES = [1, 2, 5, 31, 32, 33, 63, 64, 65, 100, 127, 150, 250, 511, 1000, 1024]


@pytest.mark.parametrize("m", SIZES)
def test_uniform_parity_all_E(F, m):
    """Every E the plain kernel serves (0..31), several tiles (n = 777, a
    ragged last CTA), three edit recipes."""
    n = 777 if m <= 256 else 260
    for name, rec in recipes().items():
        reads, refs = synth.pairs_fixed(7 + m, 0, n, m, rec)
        for E in list(range(0, 17)) + [20, 25, 31]:
            acc, obs = gpu_filter_fixed(F, reads, refs, E)
            oacc, oobs = oracle_fixed(reads, refs, E)
            assert_same(acc, obs, oacc, oobs, f"m={m} E={E} {name}")


@pytest.mark.parametrize("m", [64, 100, 200])
def test_many_tiles_per_cta_every_pair(F, m):
    """Enough pairs for every persistent CTA to cycle its shared-memory ring
    many times (with a partial last tile), every pair compared."""
    n = 1_500_001
    reads, refs = synth.pairs_fixed(55 + m, 0, n, m, synth.SHORT_POISSON)
    q = F.pack(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack(to_dev(refs.reshape(-1)), m=m, n=n)
    for E in (0, 3, 10):
        acc, obs = F.filter(q, r, m=m, e=E, n=n, sync=True)
        oacc, oobs = oracle_fixed(reads, refs, E)
        assert_same(acc.cpu().numpy(), obs.cpu().numpy(), oacc, oobs,
                    f"m={m} E={E}")


def test_unaligned_packed_input(F):
    """Packed input not 16-byte aligned: tiles are loaded without bulk
    copies."""
    torch = torch_cuda()
    n, m = 300_000, 100
    reads, refs = synth.pairs_fixed(66, 0, n, m, synth.SHORT_POISSON)
    w16 = binding.ss_packed_words(m)
    q = F.pack(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack(to_dev(refs.reshape(-1)), m=m, n=n)
    qb = torch.zeros(n * w16 + 4, dtype=torch.int32, device="cuda")
    rb = torch.zeros(n * w16 + 4, dtype=torch.int32, device="cuda")
    qb[1:1 + n * w16] = q
    rb[3:3 + n * w16] = r
    for E in (0, 2, 7):
        acc, obs = F.filter(qb[1:1 + n * w16], rb[3:3 + n * w16], m=m, e=E,
                            n=n, sync=True)
        oacc, oobs = oracle_fixed(reads, refs, E)
        assert_same(acc.cpu().numpy(), obs.cpu().numpy(), oacc, oobs,
                    f"unaligned E={E}")


def test_edge_cases(F):
    rng = np.random.default_rng(0)
    m = 100
    base = synth.pairs_fixed(9, 0, 4, m, synth.SHORT_UNIFORM_K)[0]
    allA = np.full((1, m), ord("A"), np.uint8)
    allC = np.full((1, m), ord("C"), np.uint8)
    first = base[:1].copy()
    first[0, 0] = ord("A") if first[0, 0] != ord("A") else ord("C")
    last = base[:1].copy()
    last[0, -1] = ord("A") if last[0, -1] != ord("A") else ord("C")
    reads = np.concatenate([base[:1], allA, base[:1], base[:1]])
    refs = np.concatenate([base[:1], allC, first, last])
    for E in (0, 1, 2, 5, 31):
        acc, obs = gpu_filter_fixed(F, reads, refs, E)
        oacc, oobs = oracle_fixed(reads, refs, E)
        assert_same(acc, obs, oacc, oobs, f"edges E={E}")
    # E >= m: always accepted
    for m2 in (1, 3, 7, 20):
        r, f = synth.pairs_fixed(11, 0, 200, m2, synth.SHORT_POISSON)
        for E in (m2, m2 + 1, 31):
            acc, obs = gpu_filter_fixed(F, r, f, E)
            oacc, oobs = oracle_fixed(r, f, E)
            assert_same(acc, obs, oacc, oobs, f"E>=m m={m2} E={E}")
            assert acc.all()


def test_empty_and_zero_length(F):
    torch = torch_cuda()
    z = torch.empty(0, dtype=torch.uint8, device="cuda")
    acc, obs = F.filter(z, z, m=100, e=3, n=0)
    assert acc.numel() == 0
    one = torch.zeros(8, dtype=torch.uint8, device="cuda")
    acc, obs = F.filter(one, one, m=0, e=2, n=8, fmt=FMT_ASCII, sync=True)
    assert acc.cpu().tolist() == [1] * 8 and obs.cpu().tolist() == [0] * 8


def test_binding_refuses_buffers_the_kernels_would_overrun(F):
    """A host tensor, a short buffer or a strided view never reaches a
    kernel: the binding raises before the call."""
    torch = torch_cuda()
    n, m = 1000, 100
    w16 = binding.ss_packed_words(m)
    q = torch.zeros(n * w16, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError, match="CUDA tensor"):
        F.filter(q.cpu(), q, m=m, e=3, n=n)
    with pytest.raises(ValueError, match="needs"):
        F.filter(q[:-1], q, m=m, e=3, n=n)
    with pytest.raises(ValueError, match="contiguous"):
        F.filter(q.view(n, w16).t(), q, m=m, e=3, n=n)
    with pytest.raises(ValueError, match="needs"):
        F.filter(q, q, m=m, e=3, n=n,
                 out_accept=torch.empty(n - 1, dtype=torch.uint8,
                                        device="cuda"))
    with pytest.raises(ValueError, match="needs"):
        F.filter_submaze(q, q[: w16 * (n - 1)], m=m, e=3, t=8, y=3, n=n)
    with pytest.raises(ValueError, match="host"):
        F.filter_host(q, q, m=m, e=3, n=n, fmt=FMT_PACKED2)
    acc, obs = F.filter(q, q, m=m, e=3, n=n, sync=True)  # still usable
    assert acc.all()


def test_invalid_base_through_filter(F):
    reads, refs = synth.pairs_fixed(4, 0, 300, 100, synth.SHORT_POISSON)
    refs[299, 99] = ord("x")
    with pytest.raises(binding.SSError) as ei:
        gpu_filter_fixed(F, reads, refs, 4, FMT_ASCII)
    assert ei.value.code == binding.SS_ERR_INVALID_BASE


def test_filter_host_matches_device(F):
    """ss_filter_host (host buffers, chunked copy/compute pipeline)."""
    torch = torch_cuda()
    reads, refs = synth.pairs_fixed(21, 0, 5000, 150, synth.rate_recipe(0.12))
    hq = torch.from_numpy(reads.reshape(-1).copy()).pin_memory()
    hr = torch.from_numpy(refs.reshape(-1).copy()).pin_memory()
    hq2 = hq.view(5000, 150)
    hr2 = hr.view(5000, 150)
    acc, obs = F.filter_host(hq2, hr2, m=150, e=7, fmt=FMT_ASCII)
    oacc, oobs = oracle_fixed(reads, refs, 7)
    assert_same(acc.numpy(), obs.numpy(), oacc, oobs, "filter_host")
    # a threshold sweep from packed host input, several pipeline chunks
    F2 = binding.Filter(0, workspace_bytes=1 << 20)
    try:
        dq = F2.pack(to_dev(reads.reshape(-1)), m=150, n=5000)
        drf = F2.pack(to_dev(refs.reshape(-1)), m=150, n=5000)
        F2.sync()
        pq = dq.cpu().pin_memory()
        pr = drf.cpu().pin_memory()
        sweep = [0, 3, 7, 15]
        acc, obs = F2.filter_host(pq, pr, m=150, e=sweep, n=5000,
                                  fmt=FMT_PACKED2)
        for t, E in enumerate(sweep):
            oacc, oobs = oracle_fixed(reads, refs, E)
            assert_same(acc[t].numpy(), obs[t].numpy(), oacc, oobs,
                        f"filter_host sweep E={E}")
    finally:
        F2.close()
