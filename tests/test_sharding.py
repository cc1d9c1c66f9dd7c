"""Multi-rank host logic on CPU (gloo, world size 2): beams split across
ranks with none lost or duplicated, candidate lists gathered on rank 0 in a
deterministic order, and the max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1112_0065_gb300.search import CAND_DTYPE
from paper_1112_0065_gb300.sharding import beams_of_rank


def test_round_robin_covers_every_beam_once():
    for ws in (1, 2, 3, 8, 13, 16):
        got = sorted(b for r in range(ws) for b in beams_of_rank(13, ws, r))
        assert got == list(range(13))
    with pytest.raises(ValueError):
        beams_of_rank(13, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_1112_0065_gb300.sharding import beams_of_rank, gather_candidates, max_over_ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = beams_of_rank(13, world, rank)
    c = np.zeros(len(mine) * 2, dtype=CAND_DTYPE)
    for i, b in enumerate(mine):
        for k in range(2):
            c[2 * i + k]["beam"], c[2 * i + k]["d"], c[2 * i + k]["t"] = b, 10 - k, 100 * b + k
    got = gather_candidates(c)
    slow = max_over_ranks(1.0 + rank)
    if rank == 0:
        q.put((got["beam"].tolist(), got["d"].tolist(), slow))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    beams, ds, slow = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert beams == [b for b in range(13) for _ in range(2)]
    assert ds == [9, 10] * 13
    assert slow == 2.0
