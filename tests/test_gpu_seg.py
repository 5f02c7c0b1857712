"""GPU tests of the bucketed form's first kernel (k_seg_direct): input tiles
of 128 pairs that share one length <= 256 and one threshold <= 31 over
back-to-back words are routed on the plain pipeline, every other tile goes
to the classes.  Each case is compared with the oracle pair by pair:

* segments of different (m, E) inside one CTA's group of tiles, with tile
  boundaries inside and between segments;
* the same batch with its words starting one word past a 16-byte boundary
  (the tiles staged by plain loads instead of bulk copies);
* a segment with one pair's words moved elsewhere (its tile deferred to the
  classes, the neighbouring tiles still routed directly).
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


# (pairs, m, E) segments: ragged counts so tiles straddle segments
SEGMENTS = [(700, 100, 4), (333, 150, 7), (260, 60, 20), (128, 256, 31),
            (901, 100, 0), (77, 17, 2)]


def _batch(shift_words=0, move_pair=None):
    """Concatenated packed pairs of SEGMENTS; returns device tensors and
    host data for the oracle."""
    torch = _torch()
    L = np.concatenate([np.full(k, m, np.int32) for k, m, _ in SEGMENTS])
    E = np.concatenate([np.full(k, e, np.int32) for k, _, e in SEGMENTS])
    reads, refs, off = synth.pairs_varlen(4242, 0, L, synth.rate_recipe(0.06))
    n = len(L)
    words = (L.astype(np.int64) + 15) // 16
    woff = np.zeros(n + 1, np.int64)
    np.cumsum(words, out=woff[1:])
    woff = woff + shift_words
    total = int(woff[-1]) + 64
    if move_pair is not None:
        # the pair's words go past the end of the batch: its tile is no
        # longer back to back
        woff[move_pair] = total
        total += int(words[move_pair]) + 64
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dL, dE, dwo = dev(L), dev(E), dev(woff[:n])
    pq = torch.zeros(total, dtype=torch.int32, device="cuda")
    pr = torch.zeros_like(pq)
    with binding.Filter(0) as F:
        F.pack(dev(reads), offsets=dev(off[:-1]), lengths=dL, out=pq,
               out_offsets=dwo)
        F.pack(dev(refs), offsets=dev(off[:-1]), lengths=dL, out=pr,
               out_offsets=dwo)
        F.sync()
    return pq, pr, dwo, dL, dE, (reads, refs, off, L, E)


def _check(flags=0, **kw):
    pq, pr, dwo, dL, dE, host = _batch(**kw)
    reads, refs, off, L, E = host
    oa, oo = oracle.filter_batch(reads, refs, L, E, offsets=off)
    torch = _torch()
    acc = torch.empty(len(L), dtype=torch.uint8, device="cuda")
    obs = torch.empty(len(L), dtype=torch.int32, device="cuda")
    with binding.Filter(0, workspace_bytes=1 << 30) as F:
        for _ in range(2):  # the same arguments: captured, then replayed
            acc.fill_(7)
            obs.fill_(-7)
            F.filter(pq, pr, offsets=dwo, lengths=dL, E=dE, flags=flags,
                     out_accept=acc, out_obstacles=obs, sync=True)
            a, o = acc.cpu().numpy(), obs.cpu().numpy()
            bad = np.flatnonzero((a != oa) | (o != oo))
            assert len(bad) == 0, (kw, bad[:5], a[bad[:5]], oa[bad[:5]],
                                   o[bad[:5]], oo[bad[:5]])


def test_segments_of_several_lengths_and_thresholds():
    _check()


def test_segments_direct_launches():
    _check(flags=binding.SS_FLAG_NO_GRAPH)


def test_segments_not_16_byte_aligned():
    _check(shift_words=1)


def test_one_pair_out_of_place_defers_its_tile():
    _check(move_pair=750)
