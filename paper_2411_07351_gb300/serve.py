"""Serving loop with continuous batching.

Requests (images of any size) arrive over time.  The server keeps plans in
an LRU cache and buffers in PyTorch's caching allocator, admits a request
only while the device-memory budget (output + workspace of every admitted,
unfinished request) has room, and on every turn of its loop submits the
admitted small requests that are not yet running as ONE persistent batched
launch (fht_submit) on the least busy of its streams (each stream holds up to
``max_inflight`` launches, and a batched launch goes only to a stream whose
queue can take it without the host waiting: the loop itself never blocks on
the device); a large request (at least ``plain_pixels``)
fills the GPU by itself and runs the per-image kernels instead, and so does a
small request admitted alone (``solo_plain``: three short launches finish it
sooner than a one-job persistent launch).  Batches on
different streams overlap on the device; a request that arrives while others
run joins the next batch as soon as memory and a stream are free.  Plans are
built on the library's native builder threads; requests are admitted in
arrival order among those whose plans are ready, so a plan still being built
holds up only its own request.  Latency is arrival -> the host seeing the request's completion.

``PlainServer`` is the comparison: one fht_forward per request, launched on
one stream as soon as the request's plan is ready.
"""
from __future__ import annotations

import collections
import gc
import os
import sys
import time
from dataclasses import dataclass, field

import torch

from . import _capi as C
from .batch import BATCH_GENERIC_COLS, BATCH_THREADS, BATCH_TILE_COLS, BatchQueue
from .fht import PlanBuilderPool


@dataclass
class Request:
    rid: int
    arrival: float          # seconds, on the server's clock
    image: torch.Tensor     # 2-D CUDA tensor (may be a strided view)
    out: torch.Tensor | None = None
    ws: torch.Tensor | None = None
    nbytes: int = 0         # out_bytes + ws_bytes, held from admission
    out_bytes: int = 0
    ws_bytes: int = 0
    done: float | None = None
    t_ready: float | None = None   # the serving loop saw the plan built
    t_admit: float | None = None   # admitted under the memory budget
    t_launch: float | None = None  # its launch was enqueued
    plan: object = None
    batch_size: int = 0
    plan_future: object = None


class _PlanSlot:
    """The plan of one shape, shared by every request of that shape: ready
    once the loop has polled it from the builder pool."""

    def __init__(self):
        self.plan = None
        self.error = None
        self.t_submit = time.perf_counter()
        self.times = [self.t_submit, None]  # build submitted / seen finished (perf_counter)

    def done(self) -> bool:
        return self.plan is not None or self.error is not None

    def result(self):
        if self.error is not None:
            raise self.error
        return self.plan


class PlanBuilder:
    """Plans built on the library's native worker threads (PlanBuilderPool):
    the serving thread submits a shape the first time it arrives and picks the
    finished plans up on every turn (`poll`), so it never waits for a plan it
    does not need yet and no interpreter thread competes with it while plans
    are built.  Built plans stay in an LRU cache of `capacity` shapes."""

    def __init__(self, device: int, quads: int, boundary: str, split: str, workers: int | None = None,
                 batch_below: int = 0, capacity: int = 8192):
        # plan building is the serving loop's largest stage: every core but
        # the loop's own and one spare builds plans (at most 16 threads)
        if workers is None:
            workers = max(2, min(16, (os.cpu_count() or 4) - 2))
        self.device, self.quads, self.boundary, self.split = device, quads, boundary, split
        self.batch_below = batch_below
        self.capacity = capacity
        self.pool = PlanBuilderPool(threads=workers)
        self.cache: collections.OrderedDict = collections.OrderedDict()  # shape -> ready slot
        self.pending: dict = {}  # build tag -> (shape, slot)
        self.by_shape: dict = {}  # shape -> slot still being built

    def request(self, req: "Request"):
        h, w = int(req.image.shape[0]), int(req.image.shape[1])
        k = (h, w, req.image.dtype)
        slot = self.cache.get(k)
        if slot is not None:
            self.cache.move_to_end(k)
        else:
            slot = self.by_shape.get(k)
            if slot is None:
                slot = _PlanSlot()
                # requests that will be batched get the batch tile width
                batched = h * w < self.batch_below
                tag = self.pool.submit(h, w, req.image.dtype, self.quads, self.boundary, self.split, self.device,
                                       tile_cols=BATCH_TILE_COLS if batched else 0,
                                       threads=BATCH_THREADS if batched else 0,
                                       generic_cols=BATCH_GENERIC_COLS if batched else 0)
                self.pending[tag] = (k, slot)
                self.by_shape[k] = slot
        req.plan_future = slot

    def poll(self):
        for tag, res in self.pool.poll():
            k, slot = self.pending.pop(tag)
            del self.by_shape[k]
            slot.times[1] = time.perf_counter()
            if isinstance(res, Exception):
                slot.error = res
                continue
            slot.plan = res
            self.cache[k] = slot
            while len(self.cache) > self.capacity:
                self.cache.popitem(last=False)  # dropped: requests still holding the plan keep it alive

    def close(self):
        self.pool.close()


def _ready_in_order(waiting, window: int = 256, now_fn=None):
    """Requests of the first `window` waiting ones whose plans are built, in
    arrival order (a request whose plan is still being built does not hold up
    the ones behind it).  Returns a list, so the caller may remove from `waiting`."""
    ready = []
    for k, req in enumerate(waiting):
        if k >= window:
            break
        if req.plan is None:
            if not req.plan_future.done():
                continue
            req.plan = req.plan_future.result()
            req.out_bytes = req.plan.out_elems * 4
            req.ws_bytes = max(req.plan.workspace_bytes, 256)
            req.nbytes = req.out_bytes + req.ws_bytes
            if now_fn is not None:
                req.t_ready = now_fn()
        ready.append(req)
    return ready


@dataclass
class _Batch:
    event: torch.cuda.Event
    reqs: list
    slot: int
    stream: torch.cuda.Stream = field(default=None)
    plain: bool = False


class Server:
    def __init__(self, device: int = 0, budget_bytes: int = 16 << 30, streams: int = 4, quads: int = C.FHT_QALL,
                 boundary: str = "cyclic", split: str = "T", max_batch: int = 1024, keep_outputs: bool = True,
                 max_batch_pixels: int = 16 << 20, plain_pixels: int = 1 << 20, max_inflight: int = 4,
                 solo_plain: bool = True):
        self.device = device
        self.solo_plain = solo_plain
        self.max_batch_pixels = max_batch_pixels
        self.plain_pixels = plain_pixels
        self.keep_outputs = keep_outputs
        self.budget = budget_bytes
        self.quads, self.boundary, self.split = quads, boundary, split
        self.max_batch = max_batch
        self.builder = PlanBuilder(device, quads, boundary, split, batch_below=plain_pixels)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(streams)]
        self.queues = [BatchQueue(device=device, max_jobs=max_batch, max_units=1 << 22) for _ in range(streams)]
        self.inflight = [0] * streams        # launches in flight per stream
        self.max_inflight = max_inflight
        self.by_rid: dict = {}               # running batched requests by id
        self.waiting: collections.deque = collections.deque()   # arrived, not admitted
        self.admitted: collections.deque = collections.deque()  # admitted, not launched
        self.running: list[_Batch] = []
        self.used = 0
        self.finished: list[Request] = []
        self.max_used = 0
        self.batches = 0

    def arrive(self, req: Request):
        self.builder.request(req)
        self.waiting.append(req)

    def _admit(self, now_fn=None):
        for req in _ready_in_order(self.waiting, now_fn=now_fn):
            need = req.nbytes
            if self.used + need > self.budget and self.used > 0:
                break  # memory is admitted in arrival order among ready requests
            self.waiting.remove(req)
            self.used += need
            self.max_used = max(self.max_used, self.used)
            if now_fn is not None:
                req.t_admit = now_fn()
            self.admitted.append(req)

    def _finish(self, r, t, release_ws: bool):
        # A batched request's output is complete when its flag is seen, but its
        # workspace stays allocated until the whole launch has ended: only the
        # output's bytes are released here in that case (see _retire).
        r.done = t
        self.used -= r.nbytes if release_ws else r.out_bytes
        if not self.keep_outputs:
            r.out = None
        self.finished.append(r)

    def _retire(self, now_fn):
        # batched requests finish one by one (per-job completion flags)
        for q in self.queues:
            for rid in q.poll(cap=4096):
                r = self.by_rid.pop(rid, None)
                if r is not None:
                    self._finish(r, now_fn(), release_ws=False)
        still = []
        for b in self.running:
            if b.plain:
                if b.event.query():
                    r = b.reqs[0]
                    self._finish(r, now_fn(), release_ws=True)
                    r.ws = None
                    self.inflight[b.slot] -= 1
                else:
                    still.append(b)
                continue
            # a launch's workspaces are released (and their bytes returned to
            # the budget), and its stream slot counted free, once every
            # request is done and the launch has ended
            if all(r.done is not None for r in b.reqs) and b.event.query():
                for r in b.reqs:
                    r.ws = None
                    self.used -= r.ws_bytes
                self.inflight[b.slot] -= 1
            else:
                still.append(b)
        self.running = still

    def _pick_stream(self, batched: bool):
        """The least-loaded stream with room for another launch; for a batched
        launch also one whose queue can take a submit without the host waiting
        (its previous table copies have run).  None: launch nothing this turn,
        the loop goes on retiring, polling plans and admitting."""
        best = None
        for k in range(len(self.streams)):
            if self.inflight[k] >= self.max_inflight:
                continue
            if best is not None and self.inflight[k] >= self.inflight[best]:
                continue
            if batched and not self.queues[k].ready():
                continue
            best = k
        return best

    def _launch_plain(self) -> bool:
        """Whether the head of the admitted queue runs the per-image kernels:
        a large request (it fills the GPU by itself), or, with `solo_plain`, a
        small one admitted alone (three short launches finish it sooner than a
        one-job persistent launch and its host-side listing; under load the
        queue holds several and they are batched)."""
        head = self.admitted[0]
        return head.image.numel() >= self.plain_pixels or (self.solo_plain and len(self.admitted) == 1)

    def _launch(self, now_fn=None):
        while self.admitted:
            plain = self._launch_plain()
            slot = self._pick_stream(batched=not plain)
            if slot is None:
                return
            s = self.streams[slot]
            if plain:
                # the per-image kernels, no persistent batch (a large request,
                # or a small one admitted alone)
                r = self.admitted.popleft()
                with torch.cuda.stream(s):
                    r.out = r.plan.new_output()
                    r.ws = r.plan.new_workspace()
                    r.plan.forward(r.image, r.out, r.ws, stream=s)
                    ev = torch.cuda.Event()
                    ev.record(s)
                r.batch_size = 1
                if now_fn is not None:
                    r.t_launch = now_fn()
                self.running.append(_Batch(ev, [r], slot, s, plain=True))
                self.inflight[slot] += 1
                self.batches += 1
                continue
            reqs, pix = [], 0
            while (self.admitted and len(reqs) < self.max_batch and pix < self.max_batch_pixels
                   and self.admitted[0].image.numel() < self.plain_pixels):
                r = self.admitted.popleft()
                pix += r.image.numel()
                reqs.append(r)
            with torch.cuda.stream(s):
                for r in reqs:
                    r.out = r.plan.new_output()
                    r.ws = r.plan.new_workspace()
                    r.batch_size = len(reqs)
                    self.by_rid[r.rid] = r
                self.queues[slot].submit([r.image for r in reqs], self.quads, self.boundary, self.split,
                                         outs=[r.out for r in reqs], workspaces=[r.ws for r in reqs], stream=s,
                                         tags=[r.rid for r in reqs], plans=[r.plan for r in reqs])
                ev = torch.cuda.Event()
                ev.record(s)
            if now_fn is not None:
                t = now_fn()
                for r in reqs:
                    r.t_launch = t
            self.running.append(_Batch(ev, reqs, slot, s))
            self.inflight[slot] += 1
            self.batches += 1

    def step(self, now_fn):
        self.builder.poll()
        self._retire(now_fn)
        self._admit(now_fn)
        self._launch(now_fn)

    def idle(self) -> bool:
        return not (self.waiting or self.admitted or self.running)

    def close(self):
        self.builder.close()
        for q in self.queues:
            q.close()


class PlainServer:
    """One plain fht_forward per request, launched in arrival order (among
    requests whose plans are built, as in Server) on one stream, under the same
    device-memory budget as the batched server."""

    def __init__(self, device: int = 0, budget_bytes: int = 16 << 30, quads: int = C.FHT_QALL,
                 boundary: str = "cyclic", split: str = "T", keep_outputs: bool = True):
        self.device = device
        self.budget = budget_bytes
        self.keep_outputs = keep_outputs
        self.quads, self.boundary, self.split = quads, boundary, split
        self.builder = PlanBuilder(device, quads, boundary, split)
        self.stream = torch.cuda.Stream(device=device)
        self.waiting: collections.deque = collections.deque()
        self.running: collections.deque = collections.deque()
        self.finished: list[Request] = []
        self.used = 0
        self.max_used = 0
        self.batches = 0

    def arrive(self, req: Request):
        self.builder.request(req)
        self.waiting.append(req)

    def _launch(self, now_fn=None):
        for req in _ready_in_order(self.waiting, now_fn=now_fn):
            if self.used + req.nbytes > self.budget and self.used > 0:
                return
            self.waiting.remove(req)
            self.used += req.nbytes
            self.max_used = max(self.max_used, self.used)
            if now_fn is not None:
                req.t_admit = req.t_launch = now_fn()
            p = req.plan
            with torch.cuda.stream(self.stream):
                req.out = p.new_output()
                req.ws = p.new_workspace()
                p.forward(req.image, req.out, req.ws, stream=self.stream)
                ev = torch.cuda.Event()
                ev.record(self.stream)
            req.batch_size = 1
            self.running.append((ev, req))
            self.batches += 1

    def step(self, now_fn):
        self.builder.poll()
        while self.running and self.running[0][0].query():
            ev, r = self.running.popleft()
            r.done = now_fn()
            r.ws = None
            self.used -= r.nbytes
            if not self.keep_outputs:
                r.out = None
            self.finished.append(r)
        self._launch(now_fn)

    def idle(self) -> bool:
        return not (self.running or self.waiting)

    def close(self):
        self.builder.close()


def run_stream(server, requests, switch_interval: float | None = None, disable_gc: bool = True):
    """Feed `requests` (arrival-sorted Request objects) to `server` in real time.

    The serving loop and the plan builders share the interpreter lock; the
    loop yields it on every turn, and `switch_interval` (seconds) optionally
    sets the interpreter's switch interval for the run.  `server.t0` is the
    perf_counter time of arrival 0.

    Returns (finished requests, wall seconds from the first arrival to the last completion)."""
    t0 = time.perf_counter()
    server.t0 = t0

    def now():
        return time.perf_counter() - t0

    i = 0
    n = len(requests)
    old = sys.getswitchinterval()
    if switch_interval is not None:
        sys.setswitchinterval(switch_interval)
    # the cyclic garbage collector stays off while the stream is served: a
    # full collection over tens of thousands of live requests stalls the loop
    # for tens of milliseconds (requests hold no reference cycles)
    gc_was_on = gc.isenabled()
    if disable_gc:
        gc.disable()
    try:
        while i < n or not server.idle():
            t = now()
            while i < n and requests[i].arrival <= t:
                server.arrive(requests[i])
                i += 1
            server.step(now)
            time.sleep(0)  # let a builder thread take the lock now
    finally:
        sys.setswitchinterval(old)
        if gc_was_on:
            gc.enable()
    torch.cuda.synchronize()
    end = max(r.done for r in server.finished)
    return server.finished, end - (requests[0].arrival if requests else 0.0)
