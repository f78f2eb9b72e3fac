"""Host logic for running one spectrum job across ranks (one process per GPU).

The radiation sum partitions by macro-particles: every rank accumulates the
amplitudes U, V of its own particles for all (direction, frequency) bins, and
the amplitudes of all ranks add before |.|^2 (Eq. 2).  The only exchange is one
merge of the state at readout: every rank exports its state blob
(rad_state_export), rank 0 receives them in rank order and adds them into its
own context (rad_state_merge).  Works with any torch.distributed backend
(gloo on CPU, NCCL on GPUs); nothing here runs on the data path of a step.
"""
from __future__ import annotations

from typing import Callable, Optional


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) slice of n particles for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def merge_to_root(blob: bytes, merge: Callable[[bytes], None], group=None) -> Optional[int]:
    """Send this rank's state blob to rank 0, which calls merge(blob_r) for r = 1..world-1
    in rank order (its own blob is already in its context).  Returns the number of
    merged blobs on rank 0, None elsewhere."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(blob, gathered, dst=0, group=group)
    if rank != 0:
        return None
    for r in range(1, world):
        merge(gathered[r])
    return world - 1


def max_over_ranks(x: float, device=None, group=None) -> float:
    """Largest value of x over all ranks (timing: the slowest rank decides)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
