"""Multi-process helpers for running independent replicas of the apply.

The HB apply of one batch of right-hand sides has no exchange step on one
GPU; across GPUs each rank applies the operator to its own batch (weak
scaling).  These helpers assign right-hand-side shards and reduce timings.
"""
import torch
import torch.distributed as dist


def rhs_shard(nrhs_total: int, rank: int, world: int):
    """Contiguous [begin, end) block of right-hand sides owned by ``rank``."""
    base, rem = divmod(nrhs_total, world)
    begin = rank * base + min(rank, rem)
    return begin, begin + base + (1 if rank < rem else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
