"""The N > 1 bench path on CPU: world_size-2 gloo ranks run independent replicas
(one incident direction each, no data-path collective) and the job's time is the
maximum over ranks."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 100.0 * (rank + 1)
    mx = bench.max_over_ranks(my_ms, dist, "cpu")
    ang = bench.rank_direction(rank, world)
    angs = [None] * world
    dist.all_gather_object(angs, ang)
    if rank == 0:
        out.put((mx, angs, bench.aggregate_value(world, 3, mx)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    mx, angs, val = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert mx == 200.0                          # the slower rank sets the job time
    assert len(set(angs)) == 2                  # distinct directions: independent replicas
    assert abs(val - 2 * 3 / 0.2) < 1e-12       # all solves of all ranks / max time
