"""Host-side logic of the multi-GPU runs: one process per GPU, no collective on the data path.

The systems of eq. 3 (velocity fields, right-hand sides) are independent problems, so N ranks
either run N replicas of a workload (weak scaling) or split a batch of systems between them.  A
batch is split by longest-processing-time-first over the estimated cost of each system (points x
expected iterations), the classical greedy schedule whose makespan is at most 4/3 - 1/(3N) of the
optimum.  The ranks exchange only the step time (max) and the solve counts (sum) after the timed
region, through whatever torch.distributed backend the caller initialised (NCCL on GPUs, gloo in
the CPU tests).
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple


def env_ranks() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment; (0, 1, 0) without one."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def lpt_partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Indices of `costs` per rank: items in decreasing cost (ties: lower index first) each go to
    the rank with the least load so far (ties: lower rank).  Deterministic, so every rank computes
    the same partition without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(costs[i])
    for p in parts:
        p.sort()
    return parts


def makespan(costs: Sequence[float], parts: Sequence[Sequence[int]]) -> float:
    return max((sum(float(costs[i]) for i in p) for p in parts), default=0.0)


def reduce_step(ms: float, solved: int, device=None) -> Tuple[float, int]:
    """Whole-job step time (max over ranks) and solve count (sum over ranks).  Without an
    initialised process group this is the identity."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), int(solved)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(solved)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(c.item()))


def barrier(device=None) -> None:
    """Barrier over all ranks (no-op in a single process)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if device is not None and getattr(device, "type", "cpu") == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()
