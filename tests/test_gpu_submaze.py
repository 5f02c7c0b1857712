"""Sub-maze approximate mode (Snake-on-Chip's decomposition, Section 2.5) on
the GPU against the oracle's sub-maze routine, element by element; plus the
properties the decomposition has at any size (never above the exact count;
t >= m with y > E is the exact filter)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, to_dev, torch_cuda
from paper_1910_09020_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    torch_cuda()
    f = binding.Filter(0)
    yield f
    f.close()


def run(F, reads, refs, E, t, y):
    n, m = reads.shape
    q = F.pack(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack(to_dev(refs.reshape(-1)), m=m, n=n)
    acc, obs = F.filter_submaze(q, r, m=m, e=E, t=t, y=y, n=n)
    F.sync()
    return acc.cpu().numpy(), obs.cpu().numpy()


def oracle_submaze(reads, refs, E, t, y):
    n = reads.shape[0]
    acc = np.zeros(n, np.uint8)
    obs = np.zeros(n, np.int32)
    for i in range(n):
        res = oracle.filter_submaze(reads[i].tobytes(), refs[i].tobytes(),
                                    E, t, y)
        acc[i], obs[i] = res.accept, res.obstacles
    return acc, obs


@pytest.mark.parametrize("m", [1, 31, 100, 150, 257])
@pytest.mark.parametrize("t,y", [(1, 1), (8, 3), (16, 2), (33, 1),
                                 (64, 5), (1000, 1000)])
def test_submaze_matches_oracle(F, m, t, y):
    n = 1500
    reads, refs = synth.pairs_fixed(310 + m + t, 0, n, m,
                                    synth.rate_recipe(0.1))
    for E in (0, 3, 5, 9, 31):
        acc, obs = run(F, reads, refs, E, t, y)
        oacc, oobs = oracle_submaze(reads, refs, E, t, y)
        assert_same(acc, obs, oacc, oobs, f"submaze m={m} E={E} t={t} y={y}")


def test_submaze_never_exceeds_exact_and_full_span_is_exact(F):
    n, m = 3_000_000, 100
    reads, refs = synth.pairs_fixed(4242, 0, n, m, synth.SHORT_POISSON)
    q = F.pack(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack(to_dev(refs.reshape(-1)), m=m, n=n)
    for E in (2, 6, 10):
        eacc, eobs = F.filter(q, r, m=m, e=E, n=n)
        sacc, sobs = F.filter_submaze(q, r, m=m, e=E, t=8, y=3, n=n)
        facc, fobs = F.filter_submaze(q, r, m=m, e=E, t=m, y=E + 1, n=n)
        F.sync()
        eo, so, fo = eobs.cpu().numpy(), sobs.cpu().numpy(), fobs.cpu().numpy()
        assert (so <= eo).all()
        assert (fo == eo).all()
        assert (facc.cpu().numpy() == eacc.cpu().numpy()).all()
        assert (sacc.cpu().numpy() >= eacc.cpu().numpy()).all()
        idx = np.random.default_rng(E).choice(n, 300, replace=False)
        oacc, oobs = oracle_submaze(reads[idx], refs[idx], E, 8, 3)
        assert_same(sacc.cpu().numpy()[idx], so[idx], oacc, oobs,
                    f"full-size sample E={E}")


def test_submaze_unaligned_packed_input(F):
    """Packed input not 16-byte aligned: the staged launch loads its tiles
    without bulk copies."""
    torch = torch_cuda()
    n, m = 20_000, 100
    reads, refs = synth.pairs_fixed(67, 0, n, m, synth.SHORT_POISSON)
    w16 = binding.ss_packed_words(m)
    q = F.pack(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack(to_dev(refs.reshape(-1)), m=m, n=n)
    qb = torch.zeros(n * w16 + 4, dtype=torch.int32, device="cuda")
    rb = torch.zeros(n * w16 + 4, dtype=torch.int32, device="cuda")
    qb[1:1 + n * w16] = q
    rb[3:3 + n * w16] = r
    for E in (2, 6, 10):
        acc, obs = F.filter_submaze(qb[1:1 + n * w16], rb[3:3 + n * w16],
                                    m=m, e=E, t=8, y=3, n=n)
        F.sync()
        oacc, oobs = oracle_submaze(reads, refs, E, 8, 3)
        assert_same(acc.cpu().numpy(), obs.cpu().numpy(), oacc, oobs,
                    f"unaligned E={E}")


def test_submaze_edges(F):
    torch = torch_cuda()
    empty = torch.zeros(4, dtype=torch.int32, device="cuda")
    acc, obs = F.filter_submaze(empty, empty, m=100, e=3, t=8, y=3, n=0)
    one = torch.zeros(binding.ss_packed_words(100), dtype=torch.int32,
                      device="cuda")  # one pair of 100 bp
    assert acc.numel() == 0
    reads, refs = synth.pairs_fixed(5, 0, 10, 1, synth.rate_recipe(0.5))
    acc, obs = run(F, reads, refs, 0, 1, 1)
    oacc, oobs = oracle_submaze(reads, refs, 0, 1, 1)
    assert_same(acc, obs, oacc, oobs, "m=1")
    with pytest.raises(binding.SSError):
        F.filter_submaze(one, one, m=100, e=40, t=8, y=3, n=1)
    with pytest.raises(binding.SSError):
        F.filter_submaze(one, one, m=100, e=3, t=0, y=3, n=1)
