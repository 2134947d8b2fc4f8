"""Replica sharding and max-over-ranks timing with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2009_07400_gb300 import dist as mdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = mdist.rank_info()
    mine = list(mdist.shard(257, r, w))
    t = mdist.max_over_ranks([float(rank + 1), 10.0 - rank], dist)
    gathered = [None] * w
    dist.all_gather_object(gathered, mine)
    # each rank generates its own block of the 256-replica ensemble from the
    # seeded generators, as bench.py does under torchrun
    import bench
    pos, vel, boxes, counts, _, _ = bench.make_workload("ensemble256", r, w)
    parts = [None] * w
    dist.all_gather_object(parts, (pos, vel, [list(b) for b in boxes], list(counts)))
    out[rank] = (r, w, lr, t, gathered, parts)
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    ctx = torch.multiprocessing.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    import numpy as np

    import bench
    pos, vel, boxes, counts, _, _ = bench.make_workload("ensemble256")
    for rank in range(2):
        r, w, lr, t, gathered, parts = out[rank]
        assert (r, w, lr) == (rank, 2, rank)
        assert t == [2.0, 10.0]                     # element-wise max over ranks
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(257))             # every replica exactly once
        assert abs(len(gathered[0]) - len(gathered[1])) <= 1
        # the ranks' replica blocks, in rank order, are the whole ensemble
        assert [len(p[3]) for p in parts] == [128, 128]
        assert sum(sum(p[3]) for p in parts) == sum(counts)
        assert np.array_equal(np.concatenate([p[0] for p in parts]), pos)
        assert np.array_equal(np.concatenate([p[1] for p in parts]), vel)
        assert [c for p in parts for c in p[3]] == list(counts)
        assert np.array_equal(np.array([b for p in parts for b in p[2]]), np.array(boxes))


def test_shard_single_rank():
    from paper_2009_07400_gb300 import dist as mdist
    assert list(mdist.shard(5, 0, 1)) == [0, 1, 2, 3, 4]
    assert mdist.max_over_ranks([1.0, 2.0]) == [1.0, 2.0]
