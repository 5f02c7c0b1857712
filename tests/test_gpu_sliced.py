"""GPU parity of the bit-sliced layout (SS_FMT_SLICED2): its packer against
the oracle's reference packer word for word, and the plain launch over it
against the oracle element by element, through the C ABI."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, oracle_fixed, to_dev, torch_cuda
from paper_1910_09020_gb300 import binding, synth

pytestmark = pytest.mark.gpu

SLICED = binding.SS_FMT_SLICED2


@pytest.fixture(scope="module")
def F():
    torch_cuda()
    f = binding.Filter(0)
    yield f
    f.close()


def sliced_filter(F, q, r, n, m, E, out_accept=None, out_obstacles=None):
    acc, obs = F.filter(q, r, m=m, e=E, n=n, fmt=SLICED,
                        out_accept=out_accept, out_obstacles=out_obstacles)
    F.sync()
    return acc.cpu().numpy(), obs.cpu().numpy()


@pytest.mark.parametrize("n,m", [(1, 1), (31, 3), (32, 4), (33, 5),
                                 (100, 16), (257, 17), (1000, 100),
                                 (999, 101), (300, 150), (64, 250),
                                 (40, 1000), (33, 7000), (100003, 100)])
def test_pack_sliced_matches_reference(F, n, m):
    reads, _ = synth.pairs_fixed(200 + m, 0, n, m, synth.SHORT_UNIFORM_K)
    rng = np.random.default_rng(n + m)
    lower = rng.random(reads.shape) < 0.3
    reads = np.where(lower, reads | 0x20, reads).astype(np.uint8)
    got = F.pack_sliced(to_dev(reads.reshape(-1)), m=m, n=n)
    F.sync()
    got = got.cpu().numpy().view(np.uint32)[:binding.ss_sliced_words(m, n)]
    want = oracle.pack_sliced(reads)
    assert len(got) == len(want)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (n, m, bad[:5], got[bad[:5]], want[bad[:5]])


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_pack_sliced_unaligned_input(F, shift):
    torch = torch_cuda()
    n, m = 777, 100
    reads, _ = synth.pairs_fixed(211, 0, n, m, synth.SHORT_POISSON)
    buf = torch.zeros(n * m + 16, dtype=torch.uint8, device="cuda")
    buf[shift:shift + n * m] = to_dev(reads.reshape(-1))
    got = F.pack_sliced(buf[shift:shift + n * m], m=m, n=n)
    F.sync()
    got = got.cpu().numpy().view(np.uint32)
    assert (got == oracle.pack_sliced(reads)).all()


def test_pack_sliced_flags_a_bad_base(F):
    n, m = 70, 33
    reads, _ = synth.pairs_fixed(212, 0, n, m, synth.SHORT_POISSON)
    reads[45, 32] = ord("N")
    F.pack_sliced(to_dev(reads.reshape(-1)), m=m, n=n)
    with pytest.raises(binding.SSError) as e:
        F.sync()
    assert e.value.code == binding.SS_ERR_INVALID_BASE
    F.sync()  # taken: the context stays usable


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 9, 15, 16, 31, 33, 64, 100,
                               101, 150, 250, 1000])
def test_sliced_filter_every_E(F, m):
    """Every E the sliced launch is built for, ragged last group, pairs from
    near-identical to random."""
    n = 4099 if m <= 250 else 700
    reads, refs = synth.pairs_fixed(300 + m, 0, n, m, synth.rate_recipe(0.2))
    # a quarter of the pairs unrelated (random reference)
    rnd, _ = synth.pairs_fixed(301 + m, 0, n // 4, m, synth.SHORT_POISSON)
    refs[: n // 4] = rnd
    q = F.pack_sliced(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack_sliced(to_dev(refs.reshape(-1)), m=m, n=n)
    for E in range(binding.SLICED_MAX_E + 1):
        acc, obs = sliced_filter(F, q, r, n, m, E)
        oacc, oobs = oracle_fixed(reads, refs, E)
        assert_same(acc, obs, oacc, oobs, f"sliced m={m} E={E}")


@pytest.mark.parametrize("recipe", ["poisson", "uniform_k"])
def test_sliced_filter_many_groups(F, recipe):
    """Enough groups for thousands of CTAs at the headline length."""
    n, m = 200_000, 100
    rec = synth.SHORT_POISSON if recipe == "poisson" else synth.SHORT_UNIFORM_K
    reads, refs = synth.pairs_fixed(310, 0, n, m, rec)
    q = F.pack_sliced(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack_sliced(to_dev(refs.reshape(-1)), m=m, n=n)
    for E in (0, 2, 4, 6, 8, 10, 15):
        acc, obs = sliced_filter(F, q, r, n, m, E)
        oacc, oobs = oracle_fixed(reads, refs, E)
        assert_same(acc, obs, oacc, oobs, f"{recipe} E={E}")


def test_sliced_unaligned_outputs(F):
    """Outputs not 16-byte aligned: every pair written one by one."""
    torch = torch_cuda()
    n, m = 1000, 100
    reads, refs = synth.pairs_fixed(320, 0, n, m, synth.SHORT_POISSON)
    q = F.pack_sliced(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack_sliced(to_dev(refs.reshape(-1)), m=m, n=n)
    acc_buf = torch.full((n + 16,), 7, dtype=torch.uint8, device="cuda")
    obs_buf = torch.full((n + 4,), -9, dtype=torch.int32, device="cuda")
    acc, obs = sliced_filter(F, q, r, n, m, 4, out_accept=acc_buf[3:3 + n],
                             out_obstacles=obs_buf[1:1 + n])
    oacc, oobs = oracle_fixed(reads, refs, 4)
    assert_same(acc, obs, oacc, oobs, "unaligned outputs")
    assert int(acc_buf[:3].sum()) == 21 and int(obs_buf[0]) == -9
    assert int(obs_buf[1 + n]) == -9 and int(acc_buf[3 + n]) == 7


def test_sliced_argument_errors(F):
    torch = torch_cuda()
    n, m = 64, 40
    q = torch.zeros(binding.ss_sliced_words(m, n) + 4, dtype=torch.int32,
                    device="cuda")
    acc = torch.empty(n, dtype=torch.uint8, device="cuda")
    obs = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(binding.SSError) as e:
        F.filter(q, q, m=m, e=binding.SLICED_MAX_E + 1, n=n, fmt=SLICED)
    assert e.value.code == binding.SS_ERR_UNSUPPORTED
    with pytest.raises(binding.SSError) as e:  # not 16-byte aligned
        F.filter(q[1:], q[1:], m=m, e=3, n=n, fmt=SLICED)
    assert e.value.code == binding.SS_ERR_INVALID_ARG
    with pytest.raises(binding.SSError) as e:
        F.filter(q, q, m=m, e=3, n=n, fmt=SLICED,
                 flags=binding.SS_MODE_BUCKETED)
    assert e.value.code == binding.SS_ERR_UNSUPPORTED
    Es = torch.full((n,), 3, dtype=torch.int32, device="cuda")
    with pytest.raises(binding.SSError) as e:  # per-pair thresholds
        F.filter(q, q, m=m, E=Es, n=n, fmt=SLICED)
    assert e.value.code == binding.SS_ERR_INVALID_ARG
    # m = 0: every pair accepted with no obstacle
    a, o = F.filter(q, q, m=0, e=3, n=n, fmt=SLICED, out_accept=acc,
                    out_obstacles=obs, sync=True)
    assert (a.cpu().numpy() == 1).all() and (o.cpu().numpy() == 0).all()


def test_filter_host_ascii_uses_sliced_chunks():
    """ss_filter_host from ASCII host buffers: thresholds up to 15 go through
    the sliced layout (chunks of whole groups), a sweep with a larger one
    through the pair-major form; both against the oracle, several chunks."""
    torch = torch_cuda()
    n, m = 5001, 150
    reads, refs = synth.pairs_fixed(330, 0, n, m, synth.rate_recipe(0.12))
    hq = torch.from_numpy(reads.reshape(-1).copy()).pin_memory().view(n, m)
    hr = torch.from_numpy(refs.reshape(-1).copy()).pin_memory().view(n, m)
    with binding.Filter(0, workspace_bytes=1 << 20) as F2:
        for sweep in ([0, 1, 7, 15], [3, 20]):
            acc, obs = F2.filter_host(hq, hr, m=m, e=sweep,
                                      fmt=binding.SS_FMT_ASCII)
            for t, E in enumerate(sweep):
                oacc, oobs = oracle_fixed(reads, refs, E)
                assert_same(acc[t].numpy(), obs[t].numpy(), oacc, oobs,
                            f"filter_host {sweep} E={E}")


def test_filter_batch_ascii_uses_sliced_chunks():
    """ss_filter_batch on resident ASCII with a small workspace: E from 1 to
    15 packs to the sliced layout chunk by chunk (whole groups), E = 0 the
    pair-major form."""
    n, m = 10007, 100
    reads, refs = synth.pairs_fixed(331, 0, n, m, synth.SHORT_POISSON)
    dq, dr = to_dev(reads.reshape(-1)), to_dev(refs.reshape(-1))
    with binding.Filter(0, workspace_bytes=256 << 10) as F2:
        for E in (0, 1, 5, 15):
            acc, obs = F2.filter(dq, dr, m=m, e=E, n=n,
                                 fmt=binding.SS_FMT_ASCII, sync=True)
            oacc, oobs = oracle_fixed(reads, refs, E)
            assert_same(acc.cpu().numpy(), obs.cpu().numpy(), oacc, oobs,
                        f"ascii E={E}")


@pytest.mark.parametrize("es", [[0, 2, 4, 6, 8, 10], [4, 0, 3, 1, 2, 31],
                                [2, 2, 0, 15], [3], [0, 4]])
def test_filter_sweep_sliced(F, es):
    """ss_filter_sweep over the sliced layout: the thresholds 0..4 of the
    list share one pass (duplicates after the first get their own launch),
    the others one launch each; every threshold against the oracle, n not a
    multiple of 16 (results stored one by one) and one that is."""
    for n in (10007, 4096):
        m = 100
        reads, refs = synth.pairs_fixed(340 + n, 0, n, m,
                                        synth.rate_recipe(0.08))
        q = F.pack_sliced(to_dev(reads.reshape(-1)), m=m, n=n)
        r = F.pack_sliced(to_dev(refs.reshape(-1)), m=m, n=n)
        acc, obs = F.filter_sweep(q, r, m=m, e=es, n=n, sync=True)
        acc, obs = acc.cpu().numpy(), obs.cpu().numpy()
        for t, E in enumerate(es):
            oacc, oobs = oracle_fixed(reads, refs, E)
            assert_same(acc[t], obs[t], oacc, oobs, f"sweep {es} E={E} n={n}")


def test_filter_sweep_ascii_and_packed():
    """ss_filter_sweep from resident ASCII (packed to the sliced layout chunk
    by chunk in a small workspace) and from the pair-major packed format."""
    n, m = 9001, 150
    es = [0, 2, 4, 7, 20]
    reads, refs = synth.pairs_fixed(350, 0, n, m, synth.rate_recipe(0.12))
    dq, dr = to_dev(reads.reshape(-1)), to_dev(refs.reshape(-1))
    want = [oracle_fixed(reads, refs, E) for E in es]
    with binding.Filter(0, workspace_bytes=256 << 10) as F2:
        acc, obs = F2.filter_sweep(dq, dr, m=m, e=es, n=n,
                                   fmt=binding.SS_FMT_ASCII, sync=True)
        for t, E in enumerate(es):
            assert_same(acc[t].cpu().numpy(), obs[t].cpu().numpy(), *want[t],
                        f"ascii sweep E={E}")
        pq = F2.pack(dq, m=m, n=n)
        pr = F2.pack(dr, m=m, n=n)
        acc, obs = F2.filter_sweep(pq, pr, m=m, e=es, n=n,
                                   fmt=binding.SS_FMT_PACKED2, sync=True)
        for t, E in enumerate(es):
            assert_same(acc[t].cpu().numpy(), obs[t].cpu().numpy(), *want[t],
                        f"packed sweep E={E}")


@pytest.mark.parametrize("m", [5, 8, 33, 100, 150])
def test_sliced_submaze_matches_oracle(F, m):
    """The sub-maze mode over the sliced layout against the oracle's
    sso_filter_submaze, several (t, y), and equal to the pair-major form."""
    n = 3001
    reads, refs = synth.pairs_fixed(360 + m, 0, n, m, synth.rate_recipe(0.12))
    q = F.pack_sliced(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack_sliced(to_dev(refs.reshape(-1)), m=m, n=n)
    pq = F.pack(to_dev(reads.reshape(-1)), m=m, n=n)
    pr = F.pack(to_dev(refs.reshape(-1)), m=m, n=n)
    for E, t, y in ((0, 8, 3), (4, 8, 3), (10, 8, 3), (6, 5, 1), (15, 16, 2),
                    (31, 7, 9), (3, 1000, 50)):
        acc, obs = F.filter_submaze(q, r, m=m, e=E, t=t, y=y, n=n,
                                    fmt=SLICED)
        F.sync()
        acc, obs = acc.cpu().numpy(), obs.cpu().numpy()
        for p in range(0, n, 7):
            want = oracle.filter_submaze(reads[p].tobytes(), refs[p].tobytes(),
                                         E, t, y)
            assert (bool(acc[p]), int(obs[p])) == \
                (want.accept, want.obstacles), (m, E, t, y, p)
        if min(E, m - 1) <= 31:
            pacc, pobs = F.filter_submaze(pq, pr, m=m, e=E, t=t, y=y, n=n)
            F.sync()
            assert (pacc.cpu().numpy() == acc).all()
            assert (pobs.cpu().numpy() == obs).all()
