"""Data-parallel sharding of one batch of pairs across ranks (one GPU each).

Pairs are independent problems (SneakySnake, Section 2.6), so ranks need no
exchange while filtering: a batch is split into contiguous shards of about
equal estimated cost, every rank filters its own shard on its own GPU, and
the per-pair results are gathered on rank 0 at the end.  The cost estimate of
a pair is m * (E' + 1) with E' = min(E, m - 1): the greedy visits at most
E' + 1 checkpoints and each scans O(m) columns in the worst case.
"""
from __future__ import annotations

import numpy as np


def pair_costs(lengths, E) -> np.ndarray:
    m = np.asarray(lengths, dtype=np.int64)
    e = np.minimum(np.asarray(E, dtype=np.int64), np.maximum(m - 1, 0))
    return m * (e + 1) + 1


def shard_bounds(costs, world: int) -> list[tuple[int, int]]:
    """Contiguous [begin, end) per rank with about equal total cost; every
    pair belongs to exactly one shard, in order."""
    c = np.asarray(costs, dtype=np.float64)
    n = len(c)
    if world < 1:
        raise ValueError("world must be >= 1")
    prefix = np.concatenate([[0.0], np.cumsum(c)])
    total = prefix[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(prefix, total * r / world)))
    cuts.append(n)
    cuts = np.maximum.accumulate(np.clip(cuts, 0, n))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def gather_results(acc: np.ndarray, obs: np.ndarray, bounds, group=None):
    """Gather every rank's (accept, obstacles) to rank 0 in batch order.
    Returns the full arrays on rank 0 and None elsewhere.  Uses the
    process group's backend with CPU tensors (gloo) -- a one-off gather at
    the end, not a step of the filter.  A rank that has left makes the
    others' gather raise at once; one that stays up without joining makes
    it raise after the process group's timeout (set it at
    init_process_group)."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    n_max = max(e - b for b, e in bounds)
    a = torch.zeros(n_max, dtype=torch.uint8)
    o = torch.zeros(n_max, dtype=torch.int32)
    k = len(acc)
    a[:k] = torch.from_numpy(np.asarray(acc, dtype=np.uint8))
    o[:k] = torch.from_numpy(np.asarray(obs, dtype=np.int32))
    ga = [torch.zeros_like(a) for _ in range(world)] if rank == 0 else None
    go = [torch.zeros_like(o) for _ in range(world)] if rank == 0 else None
    dist.gather(a, ga, dst=0, group=group)
    dist.gather(o, go, dst=0, group=group)
    if rank != 0:
        return None
    acc_all = np.concatenate([ga[r][: e - b].numpy()
                              for r, (b, e) in enumerate(bounds)])
    obs_all = np.concatenate([go[r][: e - b].numpy()
                              for r, (b, e) in enumerate(bounds)])
    return acc_all, obs_all
