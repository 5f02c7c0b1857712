"""GPU parity of the bucketed persistent form (mixed lengths and thresholds,
large E, long reads) against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, to_dev, torch_cuda
from paper_1910_09020_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    torch_cuda()
    f = binding.Filter(0, workspace_bytes=2 << 30)
    yield f
    f.close()


def packed_batch(F, seed, lengths, recipe):
    """ASCII pairs of the given lengths -> packed on the GPU with per-pair
    word offsets.  Returns (host reads, refs, byte offsets) and the device
    (packed reads, packed refs, word offsets, lengths)."""
    torch = torch_cuda()
    L = np.ascontiguousarray(lengths, dtype=np.int32)
    reads, refs, off = synth.pairs_varlen(seed, 0, L, recipe)
    words = (L.astype(np.int64) + 15) // 16
    woff = np.zeros(len(L) + 1, np.int64)
    np.cumsum(words, out=woff[1:])
    dL, doff, dwoff = to_dev(L), to_dev(off[:-1].copy()), to_dev(woff[:-1].copy())
    total = max(int(woff[-1]), 1)
    pq = torch.zeros(total, dtype=torch.int32, device="cuda")
    pr = torch.zeros(total, dtype=torch.int32, device="cuda")
    F.pack(to_dev(reads) if len(reads) else torch.zeros(1, dtype=torch.uint8,
                                                          device="cuda"),
           offsets=doff, lengths=dL, out=pq, out_offsets=dwoff)
    F.pack(to_dev(refs) if len(refs) else torch.zeros(1, dtype=torch.uint8,
                                                        device="cuda"),
           offsets=doff, lengths=dL, out=pr, out_offsets=dwoff)
    F.sync()
    return (reads, refs, off), (pq, pr, dwoff, dL)


def run(F, dev, Es, flags=0):
    torch = torch_cuda()
    pq, pr, dwoff, dL = dev
    dE = to_dev(np.ascontiguousarray(Es, dtype=np.int32))
    acc, obs = F.filter(pq, pr, offsets=dwoff, lengths=dL, E=dE, flags=flags)
    F.sync()
    torch.cuda.synchronize()
    return acc.cpu().numpy(), obs.cpu().numpy()


def oracle_var(host, L, Es):
    reads, refs, off = host
    return oracle.filter_batch(reads, refs, L, Es, offsets=off)


def mixed_case(rng, n):
    """Lengths and thresholds that populate every class family."""
    L, Es = [], []
    for i in range(n):
        kind = i % 6
        if kind == 0:    # short, small E: thread per pair
            m = int(rng.integers(1, 300)); E = int(rng.integers(0, 32))
        elif kind == 1:  # medium, warp per pair
            m = int(rng.integers(100, 3000)); E = int(rng.integers(32, 300))
        elif kind == 2:  # E' >= 512: CTA per pair
            m = int(rng.integers(600, 2500)); E = int(rng.integers(512, 1400))
        elif kind == 3:  # E >= m (clamped rows)
            m = int(rng.integers(1, 60)); E = m + int(rng.integers(0, 40))
        elif kind == 4:  # 5 % thresholds on log-uniform lengths
            m = int(np.exp(rng.uniform(np.log(64), np.log(4000))))
            E = m * 5 // 100
        else:            # 10 %
            m = int(np.exp(rng.uniform(np.log(100), np.log(4000))))
            E = m // 10
        L.append(m)
        Es.append(E)
    return np.array(L, np.int32), np.array(Es, np.int32)


def test_mixed_batch_all_classes(F):
    rng = np.random.default_rng(7)
    L, Es = mixed_case(rng, 600)
    host, dev = packed_batch(F, 31, L, synth.rate_recipe(0.12))
    acc, obs = run(F, dev, Es)
    oacc, oobs = oracle_var(host, L, Es)
    assert_same(acc, obs, oacc, oobs, "mixed batch")
    assert 0 < oacc.mean() < 1


@pytest.mark.parametrize("rw_max_e,k", [(15, 4), (15, 8), (15, 16),
                                        (31, 4), (31, 8), (31, 16)])
def test_tuning_never_changes_results(F, rw_max_e, k):
    rng = np.random.default_rng(8)
    L, Es = mixed_case(rng, 300)
    host, dev = packed_batch(F, 32, L, synth.rate_recipe(0.1))
    F.set_tuning(rw_max_e, k)
    try:
        acc, obs = run(F, dev, Es)
    finally:
        F.set_tuning(31, 8)
    oacc, oobs = oracle_var(host, L, Es)
    assert_same(acc, obs, oacc, oobs, f"tuning {rw_max_e},{k}")


def test_warp_classes_every_bound(F):
    """Warp-per-pair pairs (32 <= E' <= 511) in every m bound of that
    family, each bound's edges included."""
    L = np.array([2048, 2049, 3072, 3073, 4096, 4097, 6144, 6145, 8192,
                  8193, 12288, 12289, 16384, 5000, 10000], np.int32)
    Es = np.array([40, 102, 300, 153, 204, 500, 307, 33, 409, 511, 100,
                   61, 200, 250, 500], np.int32)
    host, dev = packed_batch(F, 34, L, synth.rate_recipe(0.03))
    acc, obs = run(F, dev, Es)
    oacc, oobs = oracle_var(host, L, Es)
    assert_same(acc, obs, oacc, oobs, "warp classes")


def test_long_reads(F):
    """Lengths beyond the warp kernel (m > 16384) and in every m bound of
    the CTA kernel."""
    L = np.array([20000, 30000, 17000, 70000, 100000, 16385, 40000, 131072],
                 np.int32)
    Es = np.array([2000, 300, 40, 700, 100, 1700, 33, 50], np.int32)
    host, dev = packed_batch(F, 33, L, synth.rate_recipe(0.02))
    acc, obs = run(F, dev, Es)
    oacc, oobs = oracle_var(host, L, Es)
    assert_same(acc, obs, oacc, oobs, "long reads")


def test_uniform_large_E_goes_bucketed(F):
    """Fixed stride, uniform m and E beyond the plain kernel."""
    torch = torch_cuda()
    for m, E, n in ((500, 50, 700), (1500, 600, 120), (2000, 31, 300),
                    (5000, 200, 60)):
        reads, refs = synth.pairs_fixed(40 + m, 0, n, m, synth.rate_recipe(0.1))
        q = F.pack(to_dev(reads.reshape(-1)), m=m, n=n)
        r = F.pack(to_dev(refs.reshape(-1)), m=m, n=n)
        acc, obs = F.filter(q, r, m=m, e=E, n=n, sync=True)
        oacc, oobs = oracle.filter_batch(reads, refs, m, E)
        assert_same(acc.cpu().numpy(), obs.cpu().numpy(), oacc, oobs,
                    f"uniform m={m} E={E}")
        # and through ASCII (packed in the library's workspace)
        acc2, obs2 = F.filter(to_dev(reads.reshape(-1)),
                              to_dev(refs.reshape(-1)), m=m, e=E, n=n,
                              fmt=binding.SS_FMT_ASCII, sync=True)
        assert_same(acc2.cpu().numpy(), obs2.cpu().numpy(), oacc, oobs,
                    f"uniform ascii m={m} E={E}")
    torch.cuda.synchronize()


def test_forced_bucketed_matches_plain(F):
    reads, refs = synth.pairs_fixed(50, 0, 3000, 150, synth.SHORT_POISSON)
    q = F.pack(to_dev(reads.reshape(-1)), m=150, n=3000)
    r = F.pack(to_dev(refs.reshape(-1)), m=150, n=3000)
    for E in (0, 3, 7, 15, 31):
        a1, o1 = F.filter(q, r, m=150, e=E, n=3000,
                          flags=binding.SS_MODE_PLAIN, sync=True)
        a2, o2 = F.filter(q, r, m=150, e=E, n=3000,
                          flags=binding.SS_MODE_BUCKETED, sync=True)
        assert (a1.cpu() == a2.cpu()).all() and (o1.cpu() == o2.cpu()).all()


def test_graph_replay_equals_direct_launch(F):
    rng = np.random.default_rng(9)
    L, Es = mixed_case(rng, 240)
    host, dev = packed_batch(F, 34, L, synth.rate_recipe(0.1))
    before = F.counters().graph_replays
    a1, o1 = run(F, dev, Es)             # capture + replay
    a2, o2 = run(F, dev, Es)             # replay
    a3, o3 = run(F, dev, Es, flags=binding.SS_FLAG_NO_GRAPH)
    assert F.counters().graph_replays >= before + 2
    assert (a1 == a2).all() and (o1 == o2).all()
    assert (a1 == a3).all() and (o1 == o3).all()


def test_order_invariance(F):
    """A pair's result does not depend on the rest of the batch."""
    rng = np.random.default_rng(10)
    L, Es = mixed_case(rng, 200)
    host, dev = packed_batch(F, 35, L, synth.rate_recipe(0.12))
    acc, obs = run(F, dev, Es)
    perm = rng.permutation(len(L))
    reads, refs, off = host
    Lp = L[perm]
    rp = np.concatenate([reads[off[i]:off[i] + L[i]] for i in perm])
    fp = np.concatenate([refs[off[i]:off[i] + L[i]] for i in perm])
    torch = torch_cuda()
    words = (Lp.astype(np.int64) + 15) // 16
    woff = np.zeros(len(Lp) + 1, np.int64)
    np.cumsum(words, out=woff[1:])
    boff = np.zeros(len(Lp) + 1, np.int64)
    np.cumsum(Lp, out=boff[1:])
    pq = torch.zeros(int(woff[-1]), dtype=torch.int32, device="cuda")
    pr = torch.zeros(int(woff[-1]), dtype=torch.int32, device="cuda")
    dL, dwo, dbo = to_dev(Lp), to_dev(woff[:-1].copy()), to_dev(boff[:-1].copy())
    F.pack(to_dev(rp), offsets=dbo, lengths=dL, out=pq, out_offsets=dwo)
    F.pack(to_dev(fp), offsets=dbo, lengths=dL, out=pr, out_offsets=dwo)
    acc2, obs2 = run(F, (pq, pr, dwo, dL), Es[perm])
    assert (acc2 == acc[perm]).all() and (obs2 == obs[perm]).all()


def test_invalid_and_degenerate_pairs(F):
    L = np.array([100, 0, 50, 100, 3], np.int32)
    Es = np.array([5, 4, -1, 40, 0], np.int32)
    host, dev = packed_batch(F, 36, L, synth.rate_recipe(0.05))
    torch = torch_cuda()
    pq, pr, dwoff, dL = dev
    acc, obs = F.filter(pq, pr, offsets=dwoff, lengths=dL,
                        E=to_dev(Es))
    with pytest.raises(binding.SSError) as ei:
        F.sync()
    assert ei.value.code == binding.SS_ERR_INVALID_ARG
    acc, obs = acc.cpu().numpy(), obs.cpu().numpy()
    assert (acc[1], obs[1]) == (1, 0)      # m = 0: nothing to route
    assert obs[2] == -1 and acc[2] == 0    # negative E
    ok = [0, 3, 4]
    oacc, oobs = oracle_var(host, L, np.maximum(Es, 0))
    assert_same(acc[ok], obs[ok], oacc[ok], oobs[ok], "valid pairs")


def test_too_long_is_unsupported(F):
    L = np.array([140000, 200], np.int32)
    Es = np.array([100, 10], np.int32)
    host, dev = packed_batch(F, 37, L, synth.rate_recipe(0.01))
    pq, pr, dwoff, dL = dev
    acc, obs = F.filter(pq, pr, offsets=dwoff, lengths=dL, E=to_dev(Es))
    with pytest.raises(binding.SSError) as ei:
        F.sync()
    assert ei.value.code == binding.SS_ERR_UNSUPPORTED
    obs = obs.cpu().numpy()
    assert obs[0] == -1
    oacc, oobs = oracle_var(host, L, Es)
    assert obs[1] == oobs[1]


def test_autotune_picks_a_valid_tuning(F):
    rng = np.random.default_rng(11)
    L, Es = mixed_case(rng, 300)
    host, dev = packed_batch(F, 38, L, synth.rate_recipe(0.1))
    pq, pr, dwoff, dL = dev
    rmax, k, ms = F.autotune(pq, pr, offsets=dwoff, lengths=dL,
                             E=to_dev(Es), reps=2)
    assert rmax in (15, 31) and k in (4, 8, 16) and ms > 0
    acc, obs = run(F, dev, Es)
    oacc, oobs = oracle_var(host, L, Es)
    assert_same(acc, obs, oacc, oobs, "after autotune")
    F.set_tuning(31, 8)
