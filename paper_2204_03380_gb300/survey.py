"""Shot sharding of a survey over ranks (one GPU each).

Algorithm 3's shots are independent, and its last step stacks every shot's
image into one survey image.  When the shots are sharded across ranks, each
rank stacks its own shots (rbc_image_stack / rbc_batch_rtm, in shot order) and
the survey image is the sum of those partial stacks: reduce_image() forms it
with one sum all-reduce of the fp32 interior image (NCCL on GPUs, gloo on
CPU), the only exchange of the survey.

Summation order: the survey image is sum over ranks of (sum over the rank's
shots, in shot order).  With two ranks the all-reduce returns exactly
partial_0 + partial_1 on both ranks; with more, the collective's own order
decides the last bits.  Against a single process that stacks all shots in
shot order the result differs only by fp32 rounding (at most about
(nshots - 1) ulp of sum |I_s| per node).
"""
from __future__ import annotations


def shard_shots(nshots: int, rank: int, world: int, per_step: int, steps: int, warmup: int = 0):
    """Shots of every (warm-up then timed) step on this rank: each step takes
    the next world * per_step shots of the survey, cycling, and gives rank r
    the r-th block of per_step of them, so the ranks' shots are disjoint
    within a step and together cover the survey."""
    plan = []
    for s in range(warmup + steps):
        base = (s * world + rank) * per_step
        plan.append([(base + k) % nshots for k in range(per_step)])
    return plan


def reduce_image(image, group=None):
    """Sum the ranks' partial survey images in place (every rank receives the
    survey image).  A no-op without an initialised process group of more
    than one rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(image, op=dist.ReduceOp.SUM, group=group)
    return image
