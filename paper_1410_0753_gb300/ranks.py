"""Host logic for runs on several GPUs of one node, one process per GPU.

The split step has no exchange between independent grids: a single grid runs as replicas
(one per GPU), and a batched ensemble is split by scenario, each rank advancing its own share
with no collective on the data path. The only communication is on the host side: the
maximum over ranks of a timing and the sum of the work done, through torch.distributed
(NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import numpy as np


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def world_rank():
    d = _dist()
    return (d.get_world_size(), d.get_rank()) if d else (1, 0)


def _reduce(value: float, op: str, device=None) -> float:
    d = _dist()
    if d is None:
        return float(value)
    import torch
    if device is None:
        device = "cuda" if d.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.MAX if op == "max" else d.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over the ranks (the slowest rank's time)."""
    return _reduce(value, "max", device)


def sum_over_ranks(value: float, device=None) -> float:
    """The sum over the ranks (work done by the whole job)."""
    return _reduce(value, "sum", device)


def shard_scenarios(durations, world: int, rank: int) -> np.ndarray:
    """The scenarios rank `rank` of `world` advances: longest first, each to the rank with
    the least work so far (ties to the lower rank), so that the ranks' total steps differ by
    at most the longest duration. Returns the indices, ascending."""
    durations = np.asarray(durations, np.int64)
    load = np.zeros(world, np.int64)
    owner = np.empty(len(durations), np.int64)
    for b in sorted(range(len(durations)), key=lambda i: (-durations[i], i)):
        r = int(np.argmin(load))
        owner[b] = r
        load[r] += durations[b]
    return np.flatnonzero(owner == rank)
