"""GPU accuracy harness: the banded edit-distance verifier against the
oracle's Levenshtein DP, confusion counts against numpy, and -- at the
benchmark's full size -- no false rejects (Theorem 2) on 30M pairs."""
import numpy as np
import pytest

import oracle
from gpu_util import to_dev, torch_cuda
from paper_1910_09020_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    torch_cuda()
    f = binding.Filter(0)
    yield f
    f.close()


@pytest.mark.parametrize("m", [1, 17, 33, 100, 150, 250])
def test_verifier_matches_oracle(F, m):
    n = 400
    reads, refs = synth.pairs_fixed(300 + m, 0, n, m, synth.rate_recipe(0.15))
    q = F.pack(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack(to_dev(refs.reshape(-1)), m=m, n=n)
    eds = np.array([oracle.edit_distance(reads[i].tobytes(),
                                         refs[i].tobytes()) for i in range(n)])
    for E in (0, 3, 10, 25, 31):
        got = F.edit_distance(q, r, m=m, e=E, n=n)
        F.sync()
        assert (got.cpu().numpy() == np.minimum(eds, E + 1)).all(), (m, E)


def test_confusion_counts(F):
    torch = torch_cuda()
    rng = np.random.default_rng(5)
    acc = rng.integers(0, 2, 10007).astype(np.uint8)
    ed = rng.integers(0, 12, 10007).astype(np.int32)
    got = F.confusion(to_dev(acc), to_dev(ed), e=5)
    close = ed <= 5
    want = (int(((acc == 1) & close).sum()), int(((acc == 1) & ~close).sum()),
            int(((acc == 0) & close).sum()), int(((acc == 0) & ~close).sum()))
    assert got == want


def test_no_false_rejects_full_size():
    """30M pairs x 100 bp (the headline workload), E = 0, 2, ..., 10: the
    filter never rejects a pair within E edits, and the false accept rate
    falls as the maze rows grow."""
    torch = torch_cuda()
    n, m = 30_000_000, 100
    hq = torch.empty(n * m, dtype=torch.uint8, pin_memory=True)
    hr = torch.empty(n * m, dtype=torch.uint8, pin_memory=True)
    synth.pairs_fixed(1910_09020 + 2, 0, n, m, synth.SHORT_POISSON,
                      out=(hq.numpy(), hr.numpy()))
    with binding.Filter(0) as F:
        q = F.pack(hq.cuda(), m=m, n=n)
        r = F.pack(hr.cuda(), m=m, n=n)
        for E in (0, 2, 4, 6, 8, 10):
            acc, obs = F.filter(q, r, m=m, e=E, n=n)
            ed = F.edit_distance(q, r, m=m, e=E, n=n)
            ta, fa, fr, tr = F.confusion(acc, ed, e=E)
            assert ta + fa + fr + tr == n
            assert fr == 0, (E, fr)
            assert ta > 0 and tr > 0


def _varlen_packed(F, seed, L, rate):
    torch = torch_cuda()
    reads, refs, off = synth.pairs_varlen(seed, 0, L, synth.rate_recipe(rate))
    words = (L.astype(np.int64) + 15) // 16
    woff = np.zeros(len(L) + 1, np.int64)
    np.cumsum(words, out=woff[1:])
    outs = []
    for a in (reads, refs):
        o = torch.zeros(int(woff[-1]) + 4, dtype=torch.int32, device="cuda")
        F.pack(to_dev(a), offsets=to_dev(off[:-1]), lengths=to_dev(L),
               out=o, out_offsets=to_dev(woff[:-1]))
        outs.append(o)
    return reads, refs, off, outs[0], outs[1], woff


def test_warp_verifier_matches_oracle(F):
    """The warp-per-pair verifier (E up to 511, every band width class)
    against the oracle's Levenshtein DP, per-pair lengths and thresholds."""
    rng = np.random.default_rng(41)
    n = 600
    L = synth.log_uniform(41, 0, n, 1, 1500)
    E = np.minimum(rng.integers(0, 512, n),
                   np.maximum(L // 3, rng.integers(0, 40, n))).astype(np.int32)
    E[:6] = [0, 31, 32, 63, 64, 511]
    for rate in (0.03, 0.2):
        reads, refs, off, q, r, woff = _varlen_packed(F, 41, L, rate)
        got = F.edit_distance_varlen(q, r, to_dev(woff[:-1]), to_dev(L),
                                     to_dev(E))
        F.sync()
        got = got.cpu().numpy()
        for p in range(n):
            a = reads[off[p]:off[p + 1]].tobytes()
            b = refs[off[p]:off[p + 1]].tobytes()
            want = min(oracle.edit_distance(a, b), int(E[p]) + 1)
            assert got[p] == want, (p, int(L[p]), int(E[p]), got[p], want)


def test_warp_verifier_long_pairs(F):
    L = np.array([2000, 5000, 3333], np.int32)
    E = np.array([100, 250, 511], np.int32)
    reads, refs, off, q, r, woff = _varlen_packed(F, 43, L, 0.04)
    got = F.edit_distance_varlen(q, r, to_dev(woff[:-1]), to_dev(L),
                                 to_dev(E)).cpu().numpy()
    F.sync()
    for p in range(3):
        a = reads[off[p]:off[p + 1]].tobytes()
        b = refs[off[p]:off[p + 1]].tobytes()
        assert got[p] == min(oracle.edit_distance(a, b), int(E[p]) + 1)


def test_warp_verifier_rejects_out_of_range(F):
    L = np.array([100, 100, 100], np.int32)
    reads, refs, off, q, r, woff = _varlen_packed(F, 44, L, 0.1)
    got = F.edit_distance_varlen(q, r, to_dev(woff[:-1]), to_dev(L),
                                 to_dev(np.array([5, 512, 3], np.int32)))
    with pytest.raises(binding.SSError) as ei:
        F.sync()
    assert ei.value.code == binding.SS_ERR_UNSUPPORTED
    g = got.cpu().numpy()
    assert g[1] == -1 and g[0] >= 0 and g[2] >= 0
