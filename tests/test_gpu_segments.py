"""ss_filter_segments: several uniform batches (each its own length and
threshold) filtered by one call whose launches run side by side, direct or
as a replayed CUDA graph; every pair against the oracle (Section 2.4), and
the threshold sweep's launches spread over the context's streams, inside a
caller's graph capture too."""
import numpy as np
import pytest

from gpu_util import assert_same, oracle_fixed, to_dev, torch_cuda
from paper_1910_09020_gb300 import binding, synth

pytestmark = pytest.mark.gpu

SLICED = binding.SS_FMT_SLICED2
PACKED = binding.SS_FMT_PACKED2

# (m, e, n): lengths and thresholds of the paper's short reads and beyond,
# ragged last groups, a single pair, one empty segment and one of m = 0
SHAPES = [(250, 25, 3001), (150, 15, 2999), (100, 0, 64), (33, 7, 33),
          (5, 31, 1), (120, 4, 0), (0, 3, 40), (100, 10, 5000)]


@pytest.fixture(scope="module")
def F():
    torch_cuda()
    f = binding.Filter(0)
    yield f
    f.close()


def make_segments(F, fmt, seed=700):
    segs, want = [], []
    for i, (m, e, n) in enumerate(SHAPES):
        reads, refs = synth.pairs_fixed(seed + i, 0, max(n, 1), max(m, 1),
                                        synth.rate_recipe(0.12))
        if m == 0 or n == 0:
            reads, refs = reads[:n, :0], refs[:n, :0]
        dq = to_dev(reads.reshape(-1)) if reads.size else None
        dr = to_dev(refs.reshape(-1)) if refs.size else None
        torch = torch_cuda()
        if m == 0 or n == 0:
            # a placeholder buffer: m = 0 or n = 0 reads nothing
            q = r = torch.zeros(16, dtype=torch.int32, device="cuda")
        elif fmt == SLICED:
            q, r = F.pack_sliced(dq, m=m, n=n), F.pack_sliced(dr, m=m, n=n)
        else:
            q, r = F.pack(dq, m=m, n=n), F.pack(dr, m=m, n=n)
        segs.append((q, r, m, e, n))
        if m == 0:
            want.append((np.ones(n, np.uint8), np.zeros(n, np.int32)))
        else:
            want.append(oracle_fixed(reads, refs, e))
    F.sync()
    return segs, want


def check(outs, want, what):
    for k, ((acc, obs), (oacc, oobs)) in enumerate(zip(outs, want)):
        assert_same(acc.cpu().numpy(), obs.cpu().numpy(), oacc, oobs,
                    f"{what} segment {k} {SHAPES[k]}")


@pytest.mark.parametrize("fmt", [SLICED, PACKED])
def test_segments_match_oracle(F, fmt):
    """Direct launches, then the captured graph, then its replay into
    outputs overwritten in between: every segment equal to the oracle."""
    torch = torch_cuda()
    segs, want = make_segments(F, fmt)
    check(F.filter_segments(segs, fmt=fmt, graph=False, sync=True), want,
          "direct")
    outs = F.filter_segments(segs, fmt=fmt, sync=True)
    check(outs, want, "graph")
    before = F.counters().graph_replays
    for acc, obs in outs:
        acc.fill_(9)
        obs.fill_(-7)
    torch.cuda.synchronize()
    F.filter_segments([s + (o,) for s, o in zip(segs, outs)], fmt=fmt,
                      sync=True)
    assert F.counters().graph_replays == before + 1  # replayed
    check(outs, want, "replay")


def test_segments_of_one_threshold_share_launches(F):
    """Eleven segments at E = 4 (lengths 1..400, some n not a multiple of
    32) and two at E = 9: one launch per threshold, every pair against the
    oracle."""
    torch = torch_cuda()
    shapes = [(1, 4, 70), (3, 4, 33), (16, 4, 64), (17, 4, 1), (64, 4, 500),
              (99, 4, 1031), (100, 9, 2048), (150, 4, 777), (200, 4, 96),
              (250, 9, 129), (255, 4, 4099), (256, 4, 31), (400, 4, 640)]
    segs, want = [], []
    for i, (m, e, n) in enumerate(shapes):
        reads, refs = synth.pairs_fixed(760 + i, 0, n, m,
                                        synth.rate_recipe(0.1))
        q = F.pack_sliced(to_dev(reads.reshape(-1)), m=m, n=n)
        r = F.pack_sliced(to_dev(refs.reshape(-1)), m=m, n=n)
        segs.append((q, r, m, e, n))
        want.append(oracle_fixed(reads, refs, e))
    F.sync()
    before = F.counters().launches
    outs = F.filter_segments(segs, graph=False, sync=True)
    assert F.counters().launches == before + 2
    for k, ((acc, obs), (oacc, oobs)) in enumerate(zip(outs, want)):
        assert_same(acc.cpu().numpy(), obs.cpu().numpy(), oacc, oobs,
                    f"segment {k} {shapes[k]}")


# (read length, reference length, E, n): windows longer and shorter than
# the read, E from 0 to 31, E at or above the shorter length, ragged groups
FREE = [(100, 116, 10, 3001), (100, 92, 6, 2048), (100, 108, 4, 1000),
        (150, 170, 15, 513), (250, 240, 25, 96), (33, 40, 31, 70),
        (8, 5, 6, 64), (4, 9, 2, 33), (100, 101, 0, 257), (100, 116, 10, 77)]


@pytest.mark.parametrize("fmt_graph", [False, True])
def test_segments_of_different_lengths(F, fmt_graph):
    """Reads against references of another length (reads inside flanked
    windows, cut windows, unrelated pairs) over the sliced layout, mixed
    with a segment of equal lengths: every pair equal to the oracle's
    sso_filter2 (Section 2.4's correction); segments of one threshold share
    a launch."""
    import oracle
    rng = np.random.default_rng(780)
    segs, want = [], []
    for i, (mq, mr, e, n) in enumerate(FREE):
        reads, _ = synth.pairs_fixed(790 + i, 0, n, mq, synth.rate_recipe(0.1))
        refs = synth.pairs_fixed(800 + i, 0, n, mr, synth.SHORT_POISSON)[1]
        for p in range(0, n, 2):  # the read inside random flanks, or cut
            o = int(rng.integers(0, max(mr - mq, 0) + 1))
            k = min(mq, mr - o)
            refs[p, o:o + k] = reads[p, :k]
        q = F.pack_sliced(to_dev(reads.reshape(-1)), m=mq, n=n)
        r = F.pack_sliced(to_dev(refs.reshape(-1)), m=mr, n=n)
        segs.append((q, r, (mq, mr), e, n))
        want.append(oracle.filter_unequal_batch(
            reads.reshape(-1), np.arange(n, dtype=np.int64) * mq,
            np.full(n, mq, np.int32), refs.reshape(-1),
            np.arange(n, dtype=np.int64) * mr, np.full(n, mr, np.int32), e))
    # and one of equal lengths at a threshold shared with a different-length
    # segment: the two kinds never share a launch
    reads, refs = synth.pairs_fixed(830, 0, 500, 100, synth.SHORT_POISSON)
    segs.append((F.pack_sliced(to_dev(reads.reshape(-1)), m=100, n=500),
                 F.pack_sliced(to_dev(refs.reshape(-1)), m=100, n=500), 100,
                 10, 500))
    want.append(oracle_fixed(reads, refs, 10))
    F.sync()
    outs = F.filter_segments(segs, graph=fmt_graph, sync=True)
    for k, ((acc, obs), (oacc, oobs)) in enumerate(zip(outs, want)):
        assert_same(acc.cpu().numpy(), obs.cpu().numpy(), oacc, oobs,
                    f"segment {k} {(FREE + [(100, 100, 10, 500)])[k]}")
    # pair-major input takes equal lengths only
    pk = torch_cuda().zeros(64 * 8, dtype=torch_cuda().int32, device="cuda")
    with pytest.raises(binding.SSError) as ex:
        F.filter_segments([(pk, pk, (100, 116), 3, 4)], fmt=PACKED)
    assert ex.value.code == binding.SS_ERR_UNSUPPORTED


def test_more_segments_than_a_launch_takes(F):
    """37 segments at one threshold (lengths 1..37): two launches (32 + 5),
    every pair against the oracle."""
    segs, want = [], []
    for m in range(1, 38):
        n = 33 + m
        reads, refs = synth.pairs_fixed(840 + m, 0, n, m,
                                        synth.rate_recipe(0.2))
        segs.append((F.pack_sliced(to_dev(reads.reshape(-1)), m=m, n=n),
                     F.pack_sliced(to_dev(refs.reshape(-1)), m=m, n=n), m, 3,
                     n))
        want.append(oracle_fixed(reads, refs, 3))
    F.sync()
    before = F.counters().launches
    outs = F.filter_segments(segs, graph=False, sync=True)
    assert F.counters().launches == before + 2
    for k, ((acc, obs), (oacc, oobs)) in enumerate(zip(outs, want)):
        assert_same(acc.cpu().numpy(), obs.cpu().numpy(), oacc, oobs,
                    f"segment {k} (m = {k + 1})")


def test_segments_argument_errors(F):
    """The whole table is checked before anything runs: an unsupported or
    invalid segment anywhere leaves every output untouched."""
    torch = torch_cuda()
    n, m = 64, 40
    q = torch.zeros(n * m + 4, dtype=torch.int32, device="cuda")
    acc = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
    obs = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    good = (q, q, m, 3, n, (acc, obs))

    def code(segs, fmt=SLICED, **kw):
        with pytest.raises(binding.SSError) as e:
            F.filter_segments(segs, fmt=fmt, **kw)
        return e.value.code

    big = (q, q, m, binding.SLICED_MAX_E + 1, n)
    assert code([good, big]) == binding.SS_ERR_UNSUPPORTED
    assert code([good, (q[1:], q[1:], m, 3, n)]) == binding.SS_ERR_INVALID_ARG
    assert code([good, (q, q, -1, 3, n)]) == binding.SS_ERR_INVALID_ARG
    assert code([good], fmt=binding.SS_FMT_ASCII) == binding.SS_ERR_INVALID_ARG
    pk = torch.zeros(n * binding.ss_packed_words(2000), dtype=torch.int32,
                     device="cuda")
    assert code([(pk, pk, 2000, 3, n)], fmt=PACKED) == \
        binding.SS_ERR_UNSUPPORTED
    # a null output pointer, through the raw call
    arr = (binding.Segment * 1)()
    arr[0] = binding.Segment(q.data_ptr(), q.data_ptr(), n, m, 3, None, None,
                             0)
    assert binding.ss_filter_segments(F.ctx, arr, 1, SLICED, 0, 0) == \
        binding.SS_ERR_INVALID_ARG
    assert binding.ss_filter_segments(F.ctx, arr, 1, SLICED, 1, 0) == \
        binding.SS_ERR_INVALID_ARG  # unknown flag
    F.sync()
    assert (acc.cpu().numpy() == 9).all() and (obs.cpu().numpy() == -7).all()
    # nothing to do
    assert F.filter_segments([]) == []
    assert binding.ss_filter_segments(F.ctx, None, 0, SLICED, 0, 0) == \
        binding.SS_OK


def test_sweep_lanes_inside_a_caller_graph(F):
    """ss_filter_sweep forks its launches over the context's streams and
    joins them back; captured by the caller into a CUDA graph, the fork and
    join become graph edges and the replay gives the oracle's results."""
    torch = torch_cuda()
    n, m = 5003, 100
    es = [10, 0, 2, 4, 6, 8]
    reads, refs = synth.pairs_fixed(720, 0, n, m, synth.SHORT_POISSON)
    q = F.pack_sliced(to_dev(reads.reshape(-1)), m=m, n=n)
    r = F.pack_sliced(to_dev(refs.reshape(-1)), m=m, n=n)
    acc = torch.empty((len(es), n), dtype=torch.uint8, device="cuda")
    obs = torch.empty((len(es), n), dtype=torch.int32, device="cuda")
    F.sync()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            F.filter_sweep(q, r, m=m, e=es, n=n, out_accept=acc,
                           out_obstacles=obs, stream=s)
    acc.fill_(9)
    obs.fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    for t, E in enumerate(es):
        oacc, oobs = oracle_fixed(reads, refs, E)
        assert_same(acc[t].cpu().numpy(), obs[t].cpu().numpy(), oacc, oobs,
                    f"captured sweep E={E}")
