"""Multi-GPU forms of the workloads (one process per GPU).

The method's units of work that are independent -- replicas of the batched
workload, configurations of the force-matching loss, whole copies of a
single system -- are split across ranks with no data-path collective; the
only exchanges are the final reductions of scalars or gradient vectors
(torch.distributed, any backend: NCCL between GPUs, gloo on CPU).  A single
system is not split spatially: on one box each rank runs its own replica.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_shards(sizes, nranks: int):
    """Longest-processing-time assignment: items in decreasing size, each to
    the rank with the least work so far (ties to the lower rank).  Returns a
    list of index lists, one per rank, each in decreasing size."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    heap = [(0, r) for r in range(nranks)]
    out = [[] for _ in range(nranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + sizes[i], r))
    return out


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def reduce_max(value: float, device=None) -> float:
    """Maximum of a scalar over ranks (the slowest rank's time)."""
    dist = _dist()
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(arr, device=None) -> np.ndarray:
    """Elementwise sum of a float64 vector over ranks (loss and gradient of
    configurations split across ranks)."""
    dist = _dist()
    a = np.ascontiguousarray(arr, dtype=np.float64)
    if dist is None:
        return a.copy()
    import torch
    t = torch.from_numpy(a.copy())
    if device is not None:
        t = t.to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()
