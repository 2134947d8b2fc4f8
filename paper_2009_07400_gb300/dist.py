"""Multi-GPU bookkeeping for the replica-parallel path.

The hot path shards only across independent systems (replicas): every rank
owns its own GPU and its own replicas, with no collective on the data path.
Collectives appear once, outside timed work, to take the maximum of the
ranks' timings (the whole job is as slow as its slowest rank).
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, rank: int, world: int):
    """Contiguous block of item indices owned by `rank` (sizes differ by at
    most one); the blocks of all ranks partition range(n_items)."""
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(values, dist=None, device=None):
    """Element-wise maximum of a list of floats over all ranks."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()
