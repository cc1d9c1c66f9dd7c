"""Beam sharding across GPUs: each rank (one process per GPU) takes whole
beams -- the paper's one-beam-per-GPU deployment of the 13-beam receiver --
so the data path needs no collective; only the small per-gulp candidate
lists are gathered on the host of rank 0."""
from __future__ import annotations

import numpy as np


def beams_of_rank(nbeams: int, world_size: int, rank: int) -> list[int]:
    """Round-robin assignment of beams to ranks (every beam exactly once)."""
    if world_size < 1 or not 0 <= rank < world_size or nbeams < 0:
        raise ValueError("bad sharding arguments")
    return list(range(rank, nbeams, world_size))


def gather_candidates(local, group=None, dst: int = 0):
    """Gather each rank's candidate array (a numpy structured array) on rank
    `dst`: returns the concatenation, ordered by (beam, d, t), there and None
    elsewhere.  Uses torch.distributed object gathering on the host."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    parts = [None] * world if rank == dst else None
    dist.gather_object(local, parts, dst=dst, group=group)
    if rank != dst:
        return None
    allc = np.concatenate([p for p in parts if p is not None and len(p)]) if any(
        p is not None and len(p) for p in parts) else np.zeros(0, dtype=local.dtype)
    order = np.lexsort((allc["t"], allc["d"], allc["beam"]))
    return allc[order]


def max_over_ranks(value: float, group=None) -> float:
    """The slowest rank's time (what a timed step of the whole job takes)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
