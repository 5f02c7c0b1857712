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
    32) and two at E = 9: the E = 4 ones go in two launches (8 + 3), every
    pair against the oracle."""
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
    assert F.counters().launches == before + 3
    for k, ((acc, obs), (oacc, oobs)) in enumerate(zip(outs, want)):
        assert_same(acc.cpu().numpy(), obs.cpu().numpy(), oacc, oobs,
                    f"segment {k} {shapes[k]}")


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
    arr[0] = binding.Segment(q.data_ptr(), q.data_ptr(), n, m, 3, None, None)
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
