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


def world_rank() -> tuple[int, int]:
    """(world size, rank) of the initialised process group, else (1, 0)."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def my_shard(sizes: list[tuple[int, int]], quads: int = 15) -> list[int]:
    """This rank's images (indices) of a batch: every rank computes the same
    assignment from the sizes alone, so no exchange is needed."""
    world, rank = world_rank()
    return shard(sizes, world, quads)[rank]


def route(sizes: list[tuple[int, int]], world: int, quads: int = 15) -> list[int]:
    """Rank of every request of a stream, in arrival order: each goes to the
    rank with the least work routed so far (ties to the lowest rank).  The
    rule depends only on the requests seen so far, so every rank routes the
    same stream identically without exchanging anything."""
    load = [0.0] * world
    out = []
    for h, w in sizes:
        r = min(range(world), key=lambda k: (load[k], k))
        out.append(r)
        load[r] += cost(h, w, quads)
    return out


def gather_by_index(local: dict) -> dict:
    """Merge {index: object} dictionaries from every rank (host objects; for
    checking or collecting results, not a step of the transform)."""
    world, _ = world_rank()
    if world == 1:
        return dict(local)
    parts = [None] * world
    dist.all_gather_object(parts, local)
    merged: dict = {}
    for p in parts:
        dup = merged.keys() & p.keys()
        if dup:
            raise ValueError(f"indices on more than one rank: {sorted(dup)[:5]}")
        merged.update(p)
    return merged


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
