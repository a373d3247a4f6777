"""Data-parallel sharding of the E-step over ranks (the paper runs its
algorithms over MPI on many CPUs, Sec. 1; here: torch.distributed ranks).

Points are independent in the E-step, so each rank takes a contiguous block
of the data, runs the E-step on it, and the only exchange of an EM iteration
is one sum of the sufficient statistics before the (identical, replicated)
M-step.  The benchmark's multi-GPU mode runs weak-scaling E-steps with no
collective on the data path; this module is the M-step side of that design.
"""
from __future__ import annotations


def shard_range(N: int, rank: int, world: int):
    """[begin, end) of the contiguous block of N points owned by rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    q, r = divmod(N, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def allreduce_stats(st: dict, group=None):
    """Sum every statistics tensor (At, B, scal, gsc, mca) over all ranks, in
    place (NCCL for CUDA tensors, gloo for CPU tensors)."""
    import torch.distributed as dist
    for k in ("At", "B", "scal", "gsc", "mca"):
        t = st.get(k)
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return st
