"""Data-parallel sharding of the E-step over ranks (the paper runs its
algorithms over MPI on many CPUs, Sec. 1; here: torch.distributed ranks).

Points are independent in the E-step, so each rank takes a contiguous block
of the data, runs the E-step on it, and the only exchange of an EM iteration
is one sum of the sufficient statistics before the (identical, replicated)
M-step (``EM.run(group=...)`` in api.py).  The benchmark's multi-GPU mode runs
weak-scaling E-steps with no collective on the data path.
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
    place.  With NCCL the device tensors are reduced directly; with gloo (CPU
    ranks, or several ranks sharing one GPU in tests) through host copies."""
    import torch.distributed as dist
    via_host = dist.get_backend(group) == "gloo"
    for k in ("At", "B", "scal", "gsc", "mca"):
        t = st.get(k)
        if t is None:
            continue
        if via_host and t.is_cuda:
            h = t.cpu()
            dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
            t.copy_(h)
        else:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return st


def process_group_info(group=None):
    """(rank, world size) of the calling process, (0, 1) without a process group."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)
