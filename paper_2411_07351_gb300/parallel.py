"""Data-parallel sharding across GPUs (one process per GPU).

The transform has no exchange step: images, and the quadrants of one image,
are independent.  A multi-GPU job therefore only assigns whole images to
ranks and, for reporting, takes the slowest rank's time.  There is no
collective on the data path.
"""
from __future__ import annotations

import heapq

import torch
import torch.distributed as dist


def cost(h: int, w: int, quads: int = 15) -> float:
    """Relative work of one image: pixels x tree height (Theorem 1's n^2 log n), per quadrant."""
    import math

    c = 0.0
    for q in range(4):
        if quads & (1 << q):
            n, L = (h, w) if q < 2 else (w, h)
            c += n * L * max(1.0, math.log2(max(n, 2)))
    return c


def shard(sizes: list[tuple[int, int]], world: int, quads: int = 15) -> list[list[int]]:
    """Greedy longest-processing-time assignment of images (by index) to `world` ranks."""
    order = sorted(range(len(sizes)), key=lambda i: -cost(*sizes[i], quads))
    heap = [(0.0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + cost(*sizes[i], quads), r))
    for r in range(world):
        out[r].sort()
    return out


def max_over_ranks(value: float, device: torch.device | None = None) -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device: torch.device | None = None) -> float:
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
