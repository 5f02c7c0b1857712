"""Pairs of different lengths (Section 2.4's leading/trailing correction) on
the GPU against oracle.filter_unequal, element by element."""
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


def pack_varlen(F, ascii_, off, lens):
    """Concatenated ASCII with byte offsets -> packed words with word
    offsets (device)."""
    torch = torch_cuda()
    words = (lens.astype(np.int64) + 15) // 16
    woff = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(words, out=woff[1:])
    out = torch.zeros(int(woff[-1]) + 4, dtype=torch.int32, device="cuda")
    F.pack(to_dev(ascii_ if len(ascii_) else np.zeros(1, np.uint8)),
           offsets=to_dev(off[:-1].astype(np.int64)),
           lengths=to_dev(lens.astype(np.int32)), out=out,
           out_offsets=to_dev(woff[:-1]))
    return out, woff


def run(F, data, E=None, e=0):
    reads, ro, rl, refs, fo, fl = data
    q, qw = pack_varlen(F, reads, ro, rl)
    r, rw = pack_varlen(F, refs, fo, fl)
    acc, obs = F.filter_unequal(
        q, to_dev(qw[:-1]), to_dev(rl.astype(np.int32)), r, to_dev(rw[:-1]),
        to_dev(fl.astype(np.int32)), e=e,
        E=None if E is None else to_dev(np.asarray(E, np.int32)))
    F.sync()
    return acc.cpu().numpy(), obs.cpu().numpy()


def oracle_run(data, E):
    reads, ro, rl, refs, fo, fl = data
    return oracle.filter_unequal_batch(reads, ro[:-1], rl, refs, fo[:-1], fl,
                                       E)


def same(acc, obs, oacc, oobs, what):
    bad = np.nonzero((acc != oacc) | (obs != oobs))[0]
    assert len(bad) == 0, (what, len(bad), int(bad[0]), int(obs[bad[0]]),
                           int(oobs[bad[0]]))


@pytest.mark.parametrize("m,dlo,dhi", [(37, -12, 20), (100, -8, 16),
                                       (150, -30, 40), (250, -3, 3)])
def test_unequal_parity(F, m, dlo, dhi):
    n = 20000
    for name, rec in (("poisson", synth.SHORT_POISSON),
                      ("rate10", synth.rate_recipe(0.10))):
        data = synth.pairs_unequal(70 + m, 0, n, m, rec, dlo, dhi)
        for e in (0, 3, 10, 31):
            acc, obs = run(F, data, e=e)
            oacc, oobs = oracle_run(data, e)
            same(acc, obs, oacc, oobs, f"m={m} e={e} {name}")
        Es = np.random.default_rng(m).integers(0, 32, n).astype(np.int32)
        acc, obs = run(F, data, E=Es)
        oacc, oobs = oracle_run(data, Es)
        same(acc, obs, oacc, oobs, f"m={m} per-pair E {name}")


def test_unequal_edges(F):
    # E >= the shorter length (a diagonal comparing nothing), zero lengths,
    # lengths 1, equal lengths in the same batch
    cases = [(b"ACGT", b"ACGTTTT"), (b"A", b"CCCCC"), (b"CCCCC", b"A"),
             (b"", b"ACG"), (b"ACG", b""), (b"", b""), (b"ACGTACGT", b"ACGTACGA"),
             (b"AAAA", b"CCCCCC"), (b"GATTACA" * 10, b"CC" + b"GATTACA" * 10)]
    reads = b"".join(q for q, _ in cases)
    refs = b"".join(r for _, r in cases)
    rl = np.array([len(q) for q, _ in cases], np.int32)
    fl = np.array([len(r) for _, r in cases], np.int32)
    data = (np.frombuffer(reads, np.uint8), synth.offsets_of(rl), rl,
            np.frombuffer(refs, np.uint8), synth.offsets_of(fl), fl)
    for e in (0, 1, 2, 3, 5, 31):
        acc, obs = run(F, data, e=e)
        oacc, oobs = oracle_run(data, e)
        same(acc, obs, oacc, oobs, f"edges e={e}")
    # the flanked read at E = 2 costs nothing
    acc, obs = run(F, data, e=2)
    assert obs[-1] == 0 and acc[-1] == 1


def test_unequal_invalid_and_unsupported(F):
    rl = np.array([100, 100, 50], np.int32)
    fl = np.array([100, 101, 60], np.int32)
    reads, _ = synth.pairs_fixed(3, 0, 1, 400, synth.SHORT_POISSON)
    buf = reads.reshape(-1)  # every sequence below lies inside these bytes
    # equal lengths with E = 40 need 40 rows: unsupported; the others route
    q, qw = pack_varlen(F, buf, np.array([0, 100, 200, 250]), rl)
    r, rw = pack_varlen(F, buf, np.array([0, 100, 201, 261]), fl)
    acc, obs = F.filter_unequal(q, to_dev(qw[:-1]), to_dev(rl), r,
                                to_dev(rw[:-1]), to_dev(fl),
                                E=to_dev(np.array([40, 5, 55], np.int32)))
    with pytest.raises(binding.SSError) as ei:
        F.sync()
    assert ei.value.code == binding.SS_ERR_UNSUPPORTED
    o = obs.cpu().numpy()
    assert o[0] == -1 and o[1] >= 0
    assert o[2] == 0  # E >= the shorter length: nothing to count
    # a negative length
    acc, obs = F.filter_unequal(q, to_dev(qw[:-1]),
                                to_dev(np.array([-1, 100, 50], np.int32)), r,
                                to_dev(rw[:-1]), to_dev(fl), e=3)
    with pytest.raises(binding.SSError) as ei:
        F.sync()
    assert ei.value.code == binding.SS_ERR_INVALID_ARG
    assert obs.cpu().numpy()[0] == -1


def test_unequal_full_size_sampled(F):
    n, m = 2_000_000, 100
    data = synth.pairs_unequal(4242, 0, n, m, synth.SHORT_POISSON, -8, 16)
    reads, ro, rl, refs, fo, fl = data
    for e in (2, 6, 10):
        acc, obs = run(F, data, e=e)
        idx = np.random.default_rng(e).choice(n, 400, replace=False)
        for p in idx:
            Q = reads[ro[p]:ro[p + 1]].tobytes()
            R = refs[fo[p]:fo[p + 1]].tobytes()
            res = oracle.filter_unequal(Q, R, e)
            assert (bool(acc[p]), int(obs[p])) == res, (p, e)
        # no pair is counted above E+1, and most similar pairs are accepted
        assert obs.max() <= e + 1 and obs.min() >= 0
