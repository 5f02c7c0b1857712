"""Downstream pass-through: compaction of accepted pairs (indices in order,
device count) and the dense gather of their packed sequences, against the
plain definitions (numpy flatnonzero, fancy indexing)."""
import numpy as np
import pytest

from gpu_util import to_dev, torch_cuda
from paper_1910_09020_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    torch_cuda()
    f = binding.Filter(0)
    yield f
    f.close()


@pytest.mark.parametrize("n", [0, 1, 31, 4096, 4097, 100003, 3_000_001])
def test_compact_matches_flatnonzero(F, n):
    rng = np.random.default_rng(n)
    acc = (rng.random(n) < 0.37).astype(np.uint8)
    if n > 10:
        acc[: n // 10] = 0
        acc[-5:] = 1
    idx, cnt = F.compact(to_dev(acc) if n else
                         torch_cuda().zeros(1, dtype=torch_cuda().uint8,
                                            device="cuda")[:0])
    F.sync()
    want = np.flatnonzero(acc)
    c = int(cnt.item())
    assert c == len(want)
    assert (idx[:c].cpu().numpy() == want).all()


def test_filter_compact_gather_pipeline(F):
    n, m, E = 200_000, 100, 4
    reads, refs = synth.pairs_fixed(77, 0, n, m, synth.SHORT_POISSON)
    q = F.pack(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack(to_dev(refs.reshape(-1)), m=m, n=n)
    acc, obs = F.filter(q, r, m=m, e=E, n=n)
    idx, cnt = F.compact(acc)
    gq, gr = F.gather(q, r, idx, cnt, m=m, n=n)
    F.sync()
    a = acc.cpu().numpy()
    want = np.flatnonzero(a)
    c = int(cnt.item())
    assert c == len(want) and 0 < c < n
    w16 = binding.ss_packed_words(m)
    qn = q.cpu().numpy().reshape(n, w16)
    rn = r.cpu().numpy().reshape(n, w16)
    assert (gq[: c * w16].cpu().numpy().reshape(c, w16) == qn[want]).all()
    assert (gr[: c * w16].cpu().numpy().reshape(c, w16) == rn[want]).all()
    assert (gq[c * w16:].cpu().numpy() == 0).all()
