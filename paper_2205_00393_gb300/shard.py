"""Slice sharding over ranks (one process per GPU).

The sum over slices (Sec. 2.1.1, Eq. 3) splits into independent slice ranges
(Sec. 3.1; the paper deals subtasks to processes and reduces their results
once, Sec. 6.1). Ranks take disjoint blocks of slices, each sums its blocks
locally, and the only exchange is one sum of the partial results. This module
is host logic only: the per-rank contraction is passed in, so the same code
runs over NCCL with GPU contractions or over gloo on the CPU.
"""

import numpy as np


def step_range(step, world, rank, per_step, n_slices):
    """Slice range [lo, hi) of `rank` at `step` when every step deals one block
    of `per_step` slices to each rank, blocks in rank order (wrapping at
    n_slices)."""
    lo = ((step * world + rank) * per_step) % n_slices
    return lo, min(lo + per_step, n_slices)


def rank_blocks(lo, hi, per_call, world, rank):
    """Blocks of at most `per_call` slices covering [lo, hi), dealt round-robin:
    rank r gets blocks r, r + world, r + 2 world, ... Every slice of [lo, hi)
    lands in exactly one block of exactly one rank."""
    if per_call < 1 or world < 1 or not 0 <= rank < world or hi < lo:
        raise ValueError("bad sharding arguments")
    starts = range(lo, hi, per_call)
    return [(s, min(s + per_call, hi)) for i, s in enumerate(starts) if i % world == rank]


def sharded_sum(contract, lo, hi, per_call, world=1, rank=0, group=None):
    """Sum over slices [lo, hi) split across ranks: contract(a, b) returns this
    rank's complex result for slices [a, b) (a NumPy array or a tensor); the
    partial sums are added with one all-reduce (torch.distributed, when
    world > 1). Returns the total as a complex128 NumPy array on every rank."""
    total = None
    for a, b in rank_blocks(lo, hi, per_call, world, rank):
        r = contract(a, b)
        r = r.detach().cpu().numpy() if hasattr(r, "detach") else np.asarray(r)
        r = r.astype(np.complex128)
        total = r if total is None else total + r
    if world > 1:
        import torch
        import torch.distributed as dist
        if total is None:  # this rank got no block: contribute zeros of the right shape
            probe = contract(lo, lo)
            probe = probe.detach().cpu().numpy() if hasattr(probe, "detach") else np.asarray(probe)
            total = np.zeros_like(probe, dtype=np.complex128)
        t = torch.from_numpy(np.ascontiguousarray(total).view(np.float64).copy())
        if dist.get_backend(group) == "nccl":  # NCCL reduces device tensors only
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        total = t.cpu().numpy().view(np.complex128)
    return total
