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


def _reduce_worker(rank, world, port, q):
    """Each rank stacks its own shots' images (fp32 +=, in shot order, as
    rbc_image_stack does) over a sharded pass of the survey, then the ranks
    sum their partial images with reduce_image."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    from paper_2204_03380_gb300.survey import reduce_image, shard_shots
    nshots, per_step = 48, 4
    plan = shard_shots(nshots, rank, world, per_step, steps=nshots // (per_step * world))
    partial = torch.zeros((17, 29), dtype=torch.float32)
    for step in plan:
        for s in step:
            img = np.random.default_rng(1000 + s).standard_normal((17, 29)).astype(np.float32)
            partial += torch.from_numpy(img)
    mine = partial.clone()
    reduce_image(partial)
    q.put((rank, mine.numpy(), partial.numpy(), sorted(s for step in plan for s in step)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sum_their_partial_images():
    import numpy as np
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_reduce_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict((r, (mine, red, shots)) for r, mine, red, shots in (q.get(), q.get()))
    (m0, r0, s0), (m1, r1, s1) = got[0], got[1]
    # every shot of the survey stacked exactly once
    assert not set(s0) & set(s1) and sorted(s0 + s1) == list(range(48))
    # both ranks hold the survey image, exactly partial_0 + partial_1 in fp32
    assert np.array_equal(r0, r1)
    assert np.array_equal(r0, m0 + m1)
    # one process stacking all shots in shot order differs only by rounding
    seq = np.zeros((17, 29), np.float32)
    mag = np.zeros((17, 29), np.float64)
    for s in range(48):
        img = np.random.default_rng(1000 + s).standard_normal((17, 29)).astype(np.float32)
        seq += img
        mag += np.abs(img)
    assert not np.array_equal(r0, seq)        # the orders really differ
    assert np.all(np.abs(r0.astype(np.float64) - seq) <= 47 * np.finfo(np.float32).eps * mag)
