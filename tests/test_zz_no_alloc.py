"""The allocation-free entry point ss_filter_batch_noalloc.

It exists for callers that cannot allocate device memory -- a service that
reserves all GPU memory up front through its own allocator, or a plug-in
that must stay within its host program's memory -- and keeps its scratch in
a fixed array inside the library instead of a context workspace.  These
tests call it through the C ABI and require its results to equal, bit for
bit (the tolerance of every parity test here), those of ss_filter_batch on
the same pairs, on two calls in a row that share the one scratch array.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_1910_09020_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU test without a GPU"
    return torch


def _batch(F, seed, n):
    """A packed mixed batch: per-pair lengths and thresholds across the
    thread-, warp- and CTA-per-pair classes."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    L = np.empty(n, np.int32)
    Es = np.empty(n, np.int32)
    for i in range(n):
        k = i % 4
        if k == 0:
            L[i] = rng.integers(1, 400); Es[i] = rng.integers(0, 32)
        elif k == 1:
            L[i] = rng.integers(200, 3000); Es[i] = rng.integers(32, 300)
        elif k == 2:
            L[i] = rng.integers(700, 2000); Es[i] = rng.integers(512, 900)
        else:
            L[i] = rng.integers(64, 4000); Es[i] = L[i] // 20
    reads, refs, off = synth.pairs_varlen(seed, 0, L, synth.rate_recipe(0.1))
    words = (L.astype(np.int64) + 15) // 16
    woff = np.zeros(n + 1, np.int64)
    np.cumsum(words, out=woff[1:])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dL, dwo = dev(L), dev(woff[:-1])
    pq = torch.zeros(int(woff[-1]), dtype=torch.int32, device="cuda")
    pr = torch.zeros_like(pq)
    F.pack(dev(reads), offsets=dev(off[:-1]), lengths=dL, out=pq,
           out_offsets=dwo)
    F.pack(dev(refs), offsets=dev(off[:-1]), lengths=dL, out=pr,
           out_offsets=dwo)
    F.sync()
    return pq, pr, dwo, dL, dev(Es)


def _noalloc(pq, pr, dwo, dL, dE):
    torch = _torch()
    n = dL.shape[0]
    acc = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    obs = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    stream = int(torch.cuda.current_stream().cuda_stream)
    rc = binding.ss_filter_batch_noalloc(
        pq.data_ptr(), pr.data_ptr(), dwo.data_ptr(), dL.data_ptr(), 0,
        dE.data_ptr(), 0, n, stream, acc.data_ptr(), obs.data_ptr())
    assert rc == binding.SS_OK, binding.strerror(rc)
    torch.cuda.synchronize()
    return acc.cpu().numpy(), obs.cpu().numpy()


def test_noalloc_matches_ss_filter_batch_two_calls_in_a_row():
    _torch()
    with binding.Filter(0, workspace_bytes=1 << 30) as F:
        big = _batch(F, 71, 1500)
        small = _batch(F, 72, 333)
        want = []
        for b in (big, small):
            pq, pr, dwo, dL, dE = b
            a, o = F.filter(pq, pr, offsets=dwo, lengths=dL, E=dE, sync=True)
            want.append((a.cpu().numpy(), o.cpu().numpy()))
        # two calls in a row on the shared scratch: larger, then smaller
        got = [_noalloc(*big), _noalloc(*small)]
        for (ga, go), (wa, wo) in zip(got, want):
            assert (ga == wa).all() and (go == wo).all()
        # and the first batch again after the second
        ga, go = _noalloc(*big)
        assert (ga == want[0][0]).all() and (go == want[0][1]).all()


def test_noalloc_uniform_fixed_stride():
    torch = _torch()
    with binding.Filter(0) as F:
        m, E, n = 100, 5, 4000
        reads, refs = synth.pairs_fixed(73, 0, n, m, synth.SHORT_POISSON)
        q = F.pack(torch.from_numpy(reads.reshape(-1).copy()).cuda(), m=m, n=n)
        r = F.pack(torch.from_numpy(refs.reshape(-1).copy()).cuda(), m=m, n=n)
        wa, wo = F.filter(q, r, m=m, e=E, n=n, sync=True)
        acc = torch.empty(n, dtype=torch.uint8, device="cuda")
        obs = torch.empty(n, dtype=torch.int32, device="cuda")
        for _ in range(2):
            rc = binding.ss_filter_batch_noalloc(
                q.data_ptr(), r.data_ptr(), 0, 0, m, 0, E, n,
                int(torch.cuda.current_stream().cuda_stream),
                acc.data_ptr(), obs.data_ptr())
            assert rc == binding.SS_OK
            torch.cuda.synchronize()
            assert torch.equal(acc, wa) and torch.equal(obs, wo)


def test_noalloc_rejects_batches_beyond_its_scratch():
    torch = _torch()
    x = torch.zeros(16, dtype=torch.int32, device="cuda")
    acc = torch.zeros(16, dtype=torch.uint8, device="cuda")
    obs = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = binding.ss_filter_batch_noalloc(
        x.data_ptr(), x.data_ptr(), 0, 0, 100, 0, 3,
        binding.SS_NOALLOC_MAX_PAIRS + 1, 0, acc.data_ptr(), obs.data_ptr())
    assert rc == binding.SS_ERR_OOM
