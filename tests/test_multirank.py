"""The multi-GPU path of bench.py on CPU: shots are independent (Algorithm 3's
shot loop), so N ranks shard them with no data-path collective; the only
collectives are the timing barrier and the max over ranks.  Two gloo ranks
check that every step's shots are disjoint across ranks, that the run covers
the survey, and that the max reduction picks the slowest rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    plan = bench.shot_plan(240, steps=15, warmup=0, per_step=8, rank=rank, world=world)
    flat = torch.tensor([s for step in plan for s in step], dtype=torch.int64)
    out = [torch.zeros_like(flat) for _ in range(world)]
    dist.all_gather(out, flat)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put(([o.tolist() for o in out], float(t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_the_survey():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    plans, tmax = q.get()
    assert tmax == 2.0
    per_step = 8
    for s in range(15):
        a = set(plans[0][s * per_step:(s + 1) * per_step])
        b = set(plans[1][s * per_step:(s + 1) * per_step])
        assert not (a & b)
    assert set(plans[0]) | set(plans[1]) == set(range(240))
