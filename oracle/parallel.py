"""The oracle over many independent images at once (test infrastructure).

Images are independent, so whole-workload checks (thousands of images, or a
stream of large ones) spread the single-threaded oracle over the host's
cores: one spawned process per core (spawn, never fork: the caller may
already hold a CUDA context), each running ``oracle.fht`` on its share of the
images and returning a SHA-256 digest of every exact result narrowed to
int32, the output type of the integer transform.  A caller compares digests
with those of its own outputs and recomputes any image whose digest differs
to find the first differing element.  Nothing here does any of the
transform's arithmetic itself.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import multiprocessing as mp
import os

import numpy as np


def digest(a: np.ndarray) -> str:
    """SHA-256 of an array's bytes (C order)."""
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _work(args):
    items, quads, boundary, rule = args
    import oracle

    res = []
    for k, img in items:
        out = oracle.fht(np.asarray(img, dtype=np.int64), quads, boundary, rule)
        if out.size and (out.min() < -(1 << 31) or out.max() >= (1 << 31)):
            raise OverflowError(f"image {k}: the exact result does not fit int32")
        res.append((k, digest(out.astype(np.int32))))
    return res


def int32_digests(images, quads: int, boundary: int, rule: int = 0, procs: int | None = None) -> dict[int, str]:
    """Digest of the oracle's packed output (int32) for every integer image,
    keyed by the image's index in ``images``."""
    import oracle

    oracle.build()  # the children only load the library
    procs = max(1, min(procs or os.cpu_count() or 1, len(images)))
    # size-balanced shares: largest images first, each to the lightest share
    nshare = procs * 4
    shares = [[] for _ in range(nshare)]
    load = [0] * nshare
    for k in sorted(range(len(images)), key=lambda i: -images[i].size):
        b = int(np.argmin(load))
        shares[b].append((k, images[k]))
        load[b] += images[k].size
    out: dict[int, str] = {}
    # an executor (not multiprocessing.Pool): a worker that dies raises
    # BrokenProcessPool here instead of being replaced forever
    with cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        for part in ex.map(_work, [(s, quads, boundary, rule) for s in shares if s]):
            out.update(part)
    return out
