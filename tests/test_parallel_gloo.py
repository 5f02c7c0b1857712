"""Multi-rank host logic on CPU: world_size 2 over gloo.  Each rank filters
its cost-balanced shard (the CPU oracle stands in for the rank's GPU), the
results are gathered to rank 0 and must equal a single-process run."""
import os
import socket

import numpy as np
import pytest

from paper_1910_09020_gb300 import parallel, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _batch():
    L = synth.log_uniform(123, 0, 400, 20, 600)
    E = synth.thresholds(L, 5)
    reads, refs, off = synth.pairs_varlen(124, 0, L, synth.rate_recipe(0.1))
    return reads, refs, off, L, E


def _worker(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reads, refs, off, L, E = _batch()
        bounds = parallel.shard_bounds(parallel.pair_costs(L, E), world)
        b, e = bounds[rank]
        so = off[b:e + 1] - off[b]
        acc, obs = oracle.filter_batch(reads[off[b]:off[e]],
                                       refs[off[b]:off[e]], L[b:e], E[b:e],
                                       offsets=so, threads=1)
        got = parallel.gather_results(acc, obs, bounds)
        if rank == 0:
            np.savez(out_path, acc=got[0], obs=got[1])
        else:
            assert got is None
    finally:
        dist.destroy_process_group()


def test_shard_bounds_cover_every_pair_once():
    costs = parallel.pair_costs([100, 5000, 7, 0, 250, 250], [5, 250, 1, 3, 12, 12])
    for world in (1, 2, 3, 6, 8):
        b = parallel.shard_bounds(costs, world)
        assert len(b) == world and b[0][0] == 0 and b[-1][1] == 6
        assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
    L = synth.log_uniform(5, 0, 10000, 64, 10000)
    c = parallel.pair_costs(L, synth.thresholds(L, 5))
    b = parallel.shard_bounds(c, 4)
    loads = [c[x:y].sum() for x, y in b]
    assert max(loads) < 1.05 * sum(loads) / 4 + c.max()


def test_two_ranks_gloo_gather_equals_single_process(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import oracle
    oracle.build()  # compile once before the ranks start
    out = str(tmp_path / "res.npz")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    reads, refs, off, L, E = _batch()
    acc, obs = oracle.filter_batch(reads, refs, L, E, offsets=off)
    assert (got["acc"] == acc).all() and (got["obs"] == obs).all()


def _worker_lost_rank(rank, world, port, out_path, mode):
    import datetime
    import time

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    try:
        if rank == 1:
            # leaves between steps (exits), or stays up without ever
            # joining the gather (stalls past the group's timeout)
            if mode == "stalls":
                time.sleep(8)
            return
        bounds = [(0, 5), (5, 10)]
        t0 = time.time()
        try:
            parallel.gather_results(np.ones(5, np.uint8),
                                    np.zeros(5, np.int32), bounds)
            outcome = "completed"
        except Exception as e:  # the failure the test expects
            outcome = type(e).__name__
        np.savez(out_path, outcome=outcome, seconds=time.time() - t0)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
@pytest.mark.parametrize("mode", ["exits", "stalls"])
def test_lost_rank_ends_the_gather_with_an_error(tmp_path, mode):
    """Failure detection on the host: a rank that leaves between steps, or
    never joins the gather, makes the survivor's gather fail -- at once, or
    within the process group's 5 s timeout -- instead of hanging."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "lost.npz")
    mp.spawn(_worker_lost_rank, args=(2, _free_port(), out, mode), nprocs=2,
             join=True)
    got = np.load(out)
    assert str(got["outcome"]) != "completed"
    assert float(got["seconds"]) < 30
