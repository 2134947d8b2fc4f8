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
    out[rank] = (r, w, lr, t, gathered)
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
    for rank in range(2):
        r, w, lr, t, gathered = out[rank]
        assert (r, w, lr) == (rank, 2, rank)
        assert t == [2.0, 10.0]                     # element-wise max over ranks
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(257))             # every replica exactly once
        assert abs(len(gathered[0]) - len(gathered[1])) <= 1


def test_shard_single_rank():
    from paper_2009_07400_gb300 import dist as mdist
    assert list(mdist.shard(5, 0, 1)) == [0, 1, 2, 3, 4]
    assert mdist.max_over_ranks([1.0, 2.0]) == [1.0, 2.0]
