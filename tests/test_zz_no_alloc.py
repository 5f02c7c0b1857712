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

import oracle
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
    return pq, pr, dwo, dL, dev(Es), (reads, refs, off, L, Es)


def _oracle(host):
    """The CPU oracle's (accept, obstacles) for a batch made by _batch."""
    reads, refs, off, L, Es = host
    return oracle.filter_batch(reads, refs, L, Es, offsets=off)


def _noalloc(pq, pr, dwo, dL, dE, host=None):
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
            pq, pr, dwo, dL, dE, host = b
            a, o = F.filter(pq, pr, offsets=dwo, lengths=dL, E=dE, sync=True)
            want.append((a.cpu().numpy(), o.cpu().numpy()))
            # the context path itself equals the oracle on these pairs
            oa, oo = _oracle(host)
            assert (want[-1][0] == oa).all() and (want[-1][1] == oo).all()
        # two calls in a row on the shared scratch: larger, then smaller
        got = [_noalloc(*big), _noalloc(*small)]
        for (ga, go), (wa, wo), b in zip(got, want, (big, small)):
            assert (ga == wa).all() and (go == wo).all()
            oa, oo = _oracle(b[-1])
            assert (ga == oa).all() and (go == oo).all()
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
        oa, oo = oracle.filter_batch(reads, refs, m, E)
        assert (wa.cpu().numpy() == oa).all()
        assert (wo.cpu().numpy() == oo).all()
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


def test_noalloc_marks_bad_pairs_with_minus_one():
    """A negative length, a negative threshold or a pair longer than 131072
    bases gets obstacles = -1 and accept = 0 (this entry reports no status);
    the good pairs around them still equal the oracle."""
    torch = _torch()
    with binding.Filter(0) as F:
        pq, pr, dwo, dL, dE, host = _batch(F, 74, 64)
        reads, refs, off, L, Es = host
        L2, E2 = L.copy(), Es.copy()
        L2[5] = -3          # negative length
        E2[9] = -1          # negative threshold
        # too long to stage: with E' > 31 the pair belongs to the CTA-per-
        # pair classes, which refuse lengths past 131072 before reading a
        # word (a short threshold would send it to the thread-per-pair
        # class, which reads m bases from the buffers as given)
        L2[17] = 131073
        E2[17] = 1000
        dL2 = torch.from_numpy(L2).cuda()
        dE2 = torch.from_numpy(E2).cuda()
        for _ in range(2):
            ga, go = _noalloc(pq, pr, dwo, dL2, dE2)
            bad = np.zeros(len(L), bool)
            bad[[5, 9, 17]] = True
            assert (go[bad] == -1).all() and (ga[bad] == 0).all()
            oa, oo = _oracle(host)
            assert (ga[~bad] == oa[~bad]).all() and (go[~bad] == oo[~bad]).all()
