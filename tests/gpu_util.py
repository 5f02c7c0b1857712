"""Helpers of the GPU parity tests: move generator output to the device,
call the library through the C ABI, compare with the oracle."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1910_09020_gb300 import binding, synth

FMT_ASCII = binding.SS_FMT_ASCII
FMT_PACKED2 = binding.SS_FMT_PACKED2


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test without a GPU"
    return torch


def to_dev(a: np.ndarray):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def gpu_filter_fixed(F: binding.Filter, reads: np.ndarray, refs: np.ndarray,
                     E: int, fmt: int = FMT_PACKED2, flags: int = 0):
    """reads/refs: (n, m) ASCII uint8 arrays.  For PACKED2 the pairs are
    packed on the GPU by ss_pack first.  Returns host numpy (acc, obs)."""
    torch = torch_cuda()
    n, m = reads.shape
    dq, dr = to_dev(reads.reshape(-1)), to_dev(refs.reshape(-1))
    if fmt == FMT_PACKED2:
        q = F.pack(dq, m=m, n=n)
        r = F.pack(dr, m=m, n=n)
    else:
        q, r = dq, dr
    acc, obs = F.filter(q, r, m=m, e=E, n=n, fmt=fmt, flags=flags)
    F.sync()
    torch.cuda.synchronize()
    return acc.cpu().numpy(), obs.cpu().numpy()


def oracle_fixed(reads: np.ndarray, refs: np.ndarray, E: int):
    acc, obs = oracle.filter_batch(reads, refs, reads.shape[1], E)
    return acc, obs


def assert_same(acc, obs, oacc, oobs, what=""):
    bad = np.nonzero((acc != oacc) | (obs != oobs))[0]
    if len(bad):
        i = bad[0]
        raise AssertionError(
            f"{what}: {len(bad)} of {len(acc)} pairs differ; first #{i}: "
            f"gpu=({acc[i]}, {obs[i]}) oracle=({oacc[i]}, {oobs[i]})")


def recipes():
    return {
        "uniform_k": synth.SHORT_UNIFORM_K,
        "poisson": synth.SHORT_POISSON,
        "rate12": synth.rate_recipe(0.12),
    }
