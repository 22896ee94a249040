"""Autotuner for the forward transform's launch shape.

For a size bucket it times ``fht_forward`` with each candidate (column tile
of the fused / band passes x threads per CTA x the height of the subtrees
merged in shared memory: 64-row blocks with the band + spine schedule, or 32-
and 16-row subtrees with one HBM pass per tree height above them) using CUDA
events, keeps the fastest and records it in a JSON cache keyed by (h bucket,
w bucket, dtype, quadrants, boundary, split).  The candidate (192, 256, 64) is
the register-tiled block path.  ``Plan(..., tuning="auto")`` reads the cache.
Every candidate computes the same result (the tests check this); only speed
differs.

Cache file: $FHT_TUNE_CACHE, else ~/.cache/fht_tune.json.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

import torch

from . import _capi as C

# (tile_cols, threads, fused_rows)
CANDIDATES = [(tc, th, 64) for tc in (64, 96, 128, 192, 256) for th in (256, 512)] + \
    [(128, 512, 32), (64, 512, 32), (128, 512, 16)]
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("FHT_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "fht_tune.json"))


def bucket(n: int) -> int:
    """Sizes are bucketed on a half-octave grid (64, 91, 128, 181, 256, ...)."""
    return int(round(2 ** (round(2 * math.log2(max(n, 1))) / 2)))


def key(h, w, dtype, quads, boundary, split) -> str:
    return f"{bucket(h)}x{bucket(w)}:{str(dtype).replace('torch.', '')}:q{quads}:{boundary}:{split}"


def load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(d: dict):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


PACKAGED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_table.json")


def lookup(h, w, dtype, quads, boundary, split):
    """The user's cache first, then the table shipped with the package (measured
    on GB300 by ``python -m paper_2411_07351_gb300.tune``)."""
    k = key(h, w, dtype, quads, boundary, split)
    with _lock:
        hit = load_cache().get(k)
    if hit is None and os.path.exists(PACKAGED):
        with open(PACKAGED) as f:
            hit = json.load(f).get(k)
    return hit


def sweep(sizes=(64, 128, 256, 512, 1024, 2048, 4096), dtypes=(torch.uint8, torch.float32),
          boundaries=("cyclic", "extended"), quads: int = C.FHT_QALL, reps: int = 8, out: str | None = None,
          single_quadrant_sizes=(64, 128, 256, 512)) -> dict:
    """Tune square sizes of a grid and write the winners to `out` (default: the packaged table).
    Small single-quadrant (Q0) transforms, which are latency-bound, get entries of their own."""
    table = {}
    grid = [(n, q) for n in sizes for q in (quads,)] + [(n, C.FHT_Q0) for n in single_quadrant_sizes]
    for n, q in grid:
        for dt in dtypes:
            for b in boundaries:
                e = tune(n, n, dt, q, b, "T", reps=reps, save=False)
                table[key(n, n, dt, q, b, "T")] = e
                print(key(n, n, dt, q, b, "T"), e["tile_cols"], e["threads"], e["fused_rows"], f"{e['ms']:.4f} ms",
                      flush=True)
    path = out or PACKAGED
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return table



def _time_plan(plan, x, reps: int) -> float:
    out, ws = plan.new_output(), plan.new_workspace()
    for _ in range(3):
        plan.forward(x, out, ws)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plan.forward(x, out, ws)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune(h: int, w: int, dtype=torch.float32, quads: int = C.FHT_QALL, boundary: str = "cyclic", split: str = "T",
         candidates=None, reps: int = 10, device: int | None = None, save: bool = True) -> dict:
    """Time every candidate on a seeded image of this size; return (and cache) the best."""
    from .fht import Plan

    dev = torch.cuda.current_device() if device is None else device
    g = torch.Generator(device=f"cuda:{dev}").manual_seed(1234)
    if dtype == torch.uint8:
        x = torch.randint(0, 256, (h, w), generator=g, device=f"cuda:{dev}", dtype=torch.int32).to(torch.uint8)
    elif dtype == torch.int32:
        x = torch.randint(-100, 100, (h, w), generator=g, device=f"cuda:{dev}", dtype=torch.int32)
    else:
        x = torch.randn((h, w), generator=g, device=f"cuda:{dev}", dtype=dtype)
    results = []
    for tc, th, fr in candidates or CANDIDATES:
        try:
            p = Plan(h, w, dtype, quads, boundary, split, dev, tile_cols=tc, threads=th, fused_rows=fr)
        except C.FHTError:
            continue  # e.g. too much shared memory for this dtype
        results.append((_time_plan(p, x, reps), tc, th, fr))
        p.close()
    results.sort()
    ms, tc, th, fr = results[0]
    entry = {"tile_cols": tc, "threads": th, "fused_rows": fr, "ms": ms,
             "candidates": [[r[1], r[2], r[3], r[0]] for r in results]}
    if save:
        with _lock:
            d = load_cache()
            d[key(h, w, dtype, quads, boundary, split)] = entry
            save_cache(d)
    return entry


# launch shapes of the plans of a batched launch: (tile_cols, threads, generic_cols)
BATCH_CANDIDATES = [(64, 0, 0), (96, 0, 0), (128, 0, 0), (192, 256, 32)]


def tune_batch(images, quads: int = C.FHT_QALL, boundary: str = "cyclic", split: str = "T", reps: int = 5,
               candidates=None) -> dict:
    """Time one persistent batched launch (fht_submit) over `images` with each
    candidate plan shape and return the fastest, with every candidate's time.
    The batch's own images are the workload, so the choice fits their sizes."""
    from .batch import BatchQueue

    results = []
    for shape in candidates or BATCH_CANDIDATES:
        q = BatchQueue(max_jobs=len(images), max_units=1 << 23, shape=shape)
        plans = [q.plan_for(x, quads, boundary, split) for x in images]
        outs = [p.new_output() for p in plans]
        wss = [p.new_workspace() for p in plans]
        for _ in range(2):
            q.submit(images, quads, boundary, split, outs=outs, workspaces=wss, plans=plans)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            q.submit(images, quads, boundary, split, outs=outs, workspaces=wss, plans=plans)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        results.append((statistics.median(ts), tuple(shape)))
        q.close()
        del plans, outs, wss
    results.sort()
    return {"shape": results[0][1], "ms": results[0][0], "candidates": [[list(r[1]), r[0]] for r in results]}


if __name__ == "__main__":
    import sys

    sweep(out=sys.argv[1] if len(sys.argv) > 1 else None)
