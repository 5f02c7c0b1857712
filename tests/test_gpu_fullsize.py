"""Parity at the benchmark's full sizes, in the launch configurations
bench.py times:

* 30M x 100 bp, E = 0, 2, ..., 10 (the headline sweep), over the
  bit-sliced layout as bench.py's step runs it (ss_filter_sweep: E = 0, 2,
  4 in one pass): every pair at every threshold against the oracle, and
  the pair-major plain launches equal to it;
* 10M x 250 bp + 10M x 150 bp at every E from 0 % to 10 % of the length,
  persistent: every pair against the oracle; the pair-major plain launches
  and the bit-sliced sweep over all eleven thresholds equal to it;
* the uneven 2M-pair batch (64..10000 bp, E = 5 %), one bucketed graph:
  every pair up to 2 kbp and a seeded 2 % sample of the longer ones;
* full-shape served requests (up to 4096 pairs, 100..100000 bp, E = 10 %):
  every pair up to 2 kbp and a seeded 2 % sample of the longer ones.
"""
import numpy as np
import pytest

import oracle
from paper_1910_09020_gb300 import binding, synth

pytestmark = pytest.mark.gpu

SEED = 1910_09020


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU test without a GPU"
    return torch


def _check_all(acc, obs, reads, refs, m, E, what):
    """Every pair of a fixed-length batch against the oracle."""
    oa, oo = oracle.filter_batch(reads, refs, m, E)
    bad = np.nonzero((acc != oa) | (obs != oo))[0]
    assert len(bad) == 0, (what, len(bad), bad[:5], acc[bad[:5]],
                           oa[bad[:5]], obs[bad[:5]], oo[bad[:5]])


def _check_varlen(acc, obs, idx, reads, refs, off, L, E, what):
    """Pairs idx of a concatenated batch against the oracle."""
    sub_r = np.concatenate([reads[off[i]:off[i] + L[i]] for i in idx])
    sub_f = np.concatenate([refs[off[i]:off[i] + L[i]] for i in idx])
    so = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(L[idx], out=so[1:])
    oa, oo = oracle.filter_batch(sub_r, sub_f, L[idx], E[idx], offsets=so)
    bad = np.nonzero((acc[idx] != oa) | (obs[idx] != oo))[0]
    assert len(bad) == 0, (what, len(bad), idx[bad[:5]])


def _short_and_sampled(L, seed, limit=2000, frac=0.02, at_least=0):
    """Every pair of length <= limit plus a seeded sample (frac of them,
    at least `at_least`) of the longer ones."""
    short = np.flatnonzero(L <= limit)
    long_ = np.flatnonzero(L > limit)
    k = min(len(long_), max(int(round(frac * len(long_))), at_least))
    rng = np.random.default_rng(seed)
    pick = rng.choice(long_, k, replace=False) if k else long_[:0]
    return np.sort(np.concatenate([short, pick])), len(short), k


def test_headline_sweep_30M_every_pair():
    torch = _torch()
    n, m = 30_000_000, 100
    hq = torch.empty(n * m, dtype=torch.uint8, pin_memory=True)
    hr = torch.empty(n * m, dtype=torch.uint8, pin_memory=True)
    synth.pairs_fixed(SEED + 2, 0, n, m, synth.SHORT_POISSON,
                      out=(hq.numpy(), hr.numpy()))
    reads, refs = hq.numpy().reshape(n, m), hr.numpy().reshape(n, m)
    sweep = [0, 2, 4, 6, 8, 10]
    with binding.Filter(0) as F:
        dq, dr = hq.cuda(), hr.cuda()
        sq = F.pack_sliced(dq, m=m, n=n)
        sr = F.pack_sliced(dr, m=m, n=n)
        sacc, sobs = F.filter_sweep(sq, sr, m=m, e=sweep, n=n, sync=True)
        del sq, sr
        q = F.pack(dq, m=m, n=n)
        r = F.pack(dr, m=m, n=n)
        for t, E in enumerate(sweep):
            a, o = sacc[t].cpu().numpy(), sobs[t].cpu().numpy()
            _check_all(a, o, reads, refs, m, E, f"sweep E={E}")
            acc, obs = F.filter(q, r, m=m, e=E, n=n, sync=True)
            assert (acc.cpu().numpy() == a).all(), f"pair-major E={E}"
            assert (obs.cpu().numpy() == o).all(), f"pair-major E={E}"


def test_two_lengths_20M_every_pair_both_forms():
    torch = _torch()
    n3 = 10_000_000
    rec = synth.rate_recipe(0.12)
    r250 = synth.pairs_fixed(SEED + 3, 0, n3, 250, rec)
    r150 = synth.pairs_fixed(SEED + 3, n3, n3, 150, rec)
    with binding.Filter(0, workspace_bytes=2 << 30) as F:
        bufs = []
        for (rd, rf), m in ((r250, 250), (r150, 150)):
            bufs.append((F.pack(torch.from_numpy(rd.reshape(-1)).cuda(), m=m,
                                n=n3),
                         F.pack(torch.from_numpy(rf.reshape(-1)).cuda(), m=m,
                                n=n3)))
        allq = torch.cat([bufs[0][0], bufs[1][0]])
        allr = torch.cat([bufs[0][1], bufs[1][1]])
        offs = torch.cat([torch.arange(n3, dtype=torch.int64) * 16,
                          n3 * 16 + torch.arange(n3, dtype=torch.int64) * 10]
                         ).cuda()
        lens = torch.cat([torch.full((n3,), 250, dtype=torch.int32),
                          torch.full((n3,), 150, dtype=torch.int32)]).cuda()
        # the bit-sliced sweep over all eleven thresholds of each length
        sliced = []
        for (rd, rf), m in ((r250, 250), (r150, 150)):
            sq = F.pack_sliced(torch.from_numpy(rd.reshape(-1)).cuda(), m=m,
                               n=n3)
            sr = F.pack_sliced(torch.from_numpy(rf.reshape(-1)).cuda(), m=m,
                               n=n3)
            es = [m * pct // 100 for pct in range(0, 11)]
            sa, so = F.filter_sweep(sq, sr, m=m, e=es, n=n3, sync=True)
            sliced.append((sa.cpu().numpy(), so.cpu().numpy()))
            del sq, sr, sa, so
        for pct in range(0, 11):
            e250, e150 = 250 * pct // 100, 150 * pct // 100
            a1, o1 = F.filter(bufs[0][0], bufs[0][1], m=250, e=e250, n=n3,
                              sync=True)
            a2, o2 = F.filter(bufs[1][0], bufs[1][1], m=150, e=e150, n=n3,
                              sync=True)
            Es = torch.cat([torch.full((n3,), e250, dtype=torch.int32),
                            torch.full((n3,), e150, dtype=torch.int32)]).cuda()
            ab, ob = F.filter(allq, allr, offsets=offs, lengths=lens, E=Es,
                              sync=True)
            # the persistent form against the oracle (every pair); the
            # plain form equal to it
            ab, ob = ab.cpu().numpy(), ob.cpu().numpy()
            _check_all(ab[:n3], ob[:n3], r250[0], r250[1], 250, e250,
                       f"250 bp {pct}% persistent")
            _check_all(ab[n3:], ob[n3:], r150[0], r150[1], 150, e150,
                       f"150 bp {pct}% persistent")
            assert (a1.cpu().numpy() == ab[:n3]).all(), f"250 bp {pct}%"
            assert (o1.cpu().numpy() == ob[:n3]).all(), f"250 bp {pct}%"
            assert (a2.cpu().numpy() == ab[n3:]).all(), f"150 bp {pct}%"
            assert (o2.cpu().numpy() == ob[n3:]).all(), f"150 bp {pct}%"
            for k, part in ((0, slice(0, n3)), (1, slice(n3, 2 * n3))):
                assert (sliced[k][0][pct] == ab[part]).all(), (k, pct)
                assert (sliced[k][1][pct] == ob[part]).all(), (k, pct)


def test_uneven_2M_batch_short_pairs_all_long_sampled():
    torch = _torch()
    n = 2_000_000
    L = np.sort(synth.log_uniform(SEED + 4, 0, n, 64, 10000)).astype(np.int32)
    E = synth.thresholds(L, 5)
    reads, refs, off = synth.pairs_varlen(SEED + 4, 0, L,
                                          synth.rate_recipe(0.10))
    words = (L.astype(np.int64) + 15) // 16
    woff = np.zeros(n + 1, np.int64)
    np.cumsum(words, out=woff[1:])
    with binding.Filter(0, workspace_bytes=2 << 30) as F:
        dL = torch.from_numpy(L).cuda()
        dwo = torch.from_numpy(woff[:-1].copy()).cuda()
        doff = torch.from_numpy(off[:-1].copy()).cuda()
        pq = torch.empty(int(woff[-1]), dtype=torch.int32, device="cuda")
        pr = torch.empty_like(pq)
        F.pack(torch.from_numpy(reads).cuda(), offsets=doff, lengths=dL,
               out=pq, out_offsets=dwo)
        F.pack(torch.from_numpy(refs).cuda(), offsets=doff, lengths=dL,
               out=pr, out_offsets=dwo)
        F.autotune(pq, pr, offsets=dwo, lengths=dL,
                   E=torch.from_numpy(E).cuda(), reps=1)
        acc, obs = F.filter(pq, pr, offsets=dwo, lengths=dL,
                            E=torch.from_numpy(E).cuda(), sync=True)
        acc, obs = acc.cpu().numpy(), obs.cpu().numpy()
    idx, n_short, n_long = _short_and_sampled(L, 3, at_least=5000)
    assert n_short > 1_000_000 and n_long >= 5000
    _check_varlen(acc, obs, idx, reads, refs, off, L, E, "uneven 2M")


def test_served_full_shape_requests_short_pairs_all_long_sampled():
    reqs = []
    for i in range(6):
        rng = np.random.default_rng(SEED + 5 + i)
        n = int(np.exp(rng.uniform(0, np.log(4096))))
        L = synth.log_uniform(SEED + 5000 + i, 0, n, 100, 100000)
        E = synth.thresholds(L, 10)
        reads, refs, off = synth.pairs_varlen(SEED + 50000 + i, 0, L,
                                              synth.rate_recipe(0.15))
        reqs.append((reads, refs, L, E, off))
    with binding.Server(0, hbm_budget_bytes=16 << 30, slots=2) as S:
        ts = [S.submit(r[0], r[1], r[2], r[3]) for r in reqs]
        outs = []
        for t in ts:
            assert S.wait(t) == binding.SS_OK
            outs.append(S.fetch(t))
    for k, ((rc, acc, obs, _), (reads, refs, L, E, off)) in enumerate(
            zip(outs, reqs)):
        assert rc == binding.SS_OK
        # every pair up to 2 kbp, 2 % of the longer ones (at least one)
        idx, _, _ = _short_and_sampled(np.asarray(L), 40 + k, at_least=1)
        _check_varlen(acc, obs, idx, reads, refs, off, np.asarray(L),
                      np.asarray(E), f"request {k}")
