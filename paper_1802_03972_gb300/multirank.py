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

import struct
from typing import Callable, Optional

import numpy as np

# The state blob of rad_state_export (include/rad.h): a 40-byte little-endian
# header, then the accumulators.  Header fields: magic "RADS", format version,
# precision (0 mixed, 1 FP64), n_omega, n_dir, number of component arrays,
# element size in bytes, a reserved word and the payload size in bytes.  A mixed
# payload is float32 [n_comp][n_dir * n_omega]: the compensated sums of the
# components, then their compensations (the value is sum - compensation; the
# literal sum's 8 arrays follow the main 16 when present).  An FP64 payload is
# float64 [12][n_dir * n_omega] plain sums.
BLOB_MAGIC, BLOB_VERSION = 0x52414453, 1
_HEADER = struct.Struct("<IIiiiiiiQ")


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


def parse_state_blob(blob: bytes) -> tuple[dict, np.ndarray]:
    """Header fields and payload (as [n_comp][n_bins] array) of a state blob.
    Raises ValueError for a blob that is not one (magic, version, sizes)."""
    if len(blob) < _HEADER.size:
        raise ValueError("state blob shorter than its header")
    magic, version, prec, n_omega, n_dir, n_comp, elem, _, payload = _HEADER.unpack_from(blob)
    if magic != BLOB_MAGIC or version != BLOB_VERSION:
        raise ValueError("not a version-1 radiation state blob")
    dtype = {4: np.float32, 8: np.float64}.get(elem)
    n_bins = n_omega * n_dir
    if dtype is None or n_bins < 1 or payload != n_comp * n_bins * elem or \
            len(blob) < _HEADER.size + payload:
        raise ValueError("inconsistent state blob header")
    arr = np.frombuffer(blob, dtype=dtype, count=n_comp * n_bins, offset=_HEADER.size)
    head = {"prec": prec, "n_omega": n_omega, "n_dir": n_dir, "n_comp": n_comp, "elem_size": elem}
    return head, arr.reshape(n_comp, n_bins)


def make_state_blob(head: dict, payload: np.ndarray) -> bytes:
    """A state blob from header fields and a [n_comp][n_bins] payload."""
    dtype = np.float32 if head["elem_size"] == 4 else np.float64
    arr = np.ascontiguousarray(payload, dtype=dtype)
    return _HEADER.pack(BLOB_MAGIC, BLOB_VERSION, head["prec"], head["n_omega"], head["n_dir"],
                        arr.shape[0], head["elem_size"], 0, arr.nbytes) + arr.tobytes()


def merge_state_blobs(dst: bytes, src: bytes) -> bytes:
    """Host-side counterpart of rad_state_merge: the amplitudes of `src` added to
    those of `dst` (same grid and precision), for merging ranks' states where no
    GPU is at hand.  Mixed blobs: every (sum, compensation) pair of dst takes
    src's value sum - compensation by a compensated float32 add; FP64 blobs add."""
    hd, a = parse_state_blob(dst)
    hs, b = parse_state_blob(src)
    if hd != hs:
        raise ValueError("state blobs of different grids or precisions")
    if hd["elem_size"] == 8:
        return make_state_blob(hd, a + b)
    out = a.copy()
    groups = [(0, 8)] + ([(16, 4)] if hd["n_comp"] == 24 else [])
    with np.errstate(over="ignore", invalid="ignore"):
        for base, n in groups:
            s, c = out[base:base + n], out[base + n:base + 2 * n]
            x = b[base:base + n] - b[base + n:base + 2 * n]
            y = x - c
            tt = s + y
            c[...] = (tt - s) - y
            s[...] = tt
    return make_state_blob(hd, out)
