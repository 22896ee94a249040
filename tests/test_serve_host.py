"""Host logic of the serving loop (CPU only): readiness and admission.

Requests are admitted in arrival order among those whose plans are built,
while the device-memory budget (output + workspace of every admitted,
unfinished request) has room; a request whose plan is still being built
holds up only itself, and a request larger than the whole budget still runs
when nothing else holds memory.  Plans and requests are stand-ins here: no
GPU call is made.
"""
import collections
import concurrent.futures as cf
from types import SimpleNamespace

from paper_2411_07351_gb300 import serve


def _req(rid, out_elems, ws_bytes, ready=True):
    f = cf.Future()
    if ready:
        f.set_result(SimpleNamespace(out_elems=out_elems, workspace_bytes=ws_bytes))
    return serve.Request(rid=rid, arrival=float(rid), image=None, plan_future=f)


def _server(budget):
    s = serve.Server.__new__(serve.Server)  # admission state only, no streams or queues
    s.waiting = collections.deque()
    s.admitted = collections.deque()
    s.used = 0
    s.max_used = 0
    s.budget = budget
    return s


def test_ready_in_order_skips_unbuilt_plans():
    a, b, c = _req(0, 10, 600), _req(1, 10, 600, ready=False), _req(2, 5, 0)
    got = serve._ready_in_order(collections.deque([a, b, c]))
    assert [r.rid for r in got] == [0, 2]
    assert a.nbytes == 10 * 4 + 600
    assert c.nbytes == 5 * 4 + 256  # workspaces are at least 256 bytes
    assert b.plan is None


def test_ready_in_order_window():
    reqs = [_req(k, 1, 256) for k in range(10)]
    got = serve._ready_in_order(collections.deque(reqs), window=4)
    assert [r.rid for r in got] == [0, 1, 2, 3]


def test_admission_respects_budget_and_order():
    s = _server(budget=2000)
    reqs = [_req(k, 100, 600) for k in range(5)]  # 1000 bytes each
    s.waiting.extend(reqs)
    s._admit()
    assert [r.rid for r in s.admitted] == [0, 1]
    assert s.used == 2000 and s.max_used == 2000
    assert [r.rid for r in s.waiting] == [2, 3, 4]
    # a finished request frees its bytes; the next one in order is admitted
    s.used -= reqs[0].nbytes
    s._admit()
    assert [r.rid for r in s.admitted] == [0, 1, 2]
    assert s.used == 2000


def test_unbuilt_plan_does_not_hold_up_later_requests():
    s = _server(budget=10_000)
    slow = _req(0, 100, 100, ready=False)
    fast = [_req(k, 100, 100) for k in (1, 2)]
    s.waiting.extend([slow] + fast)
    s._admit()
    assert [r.rid for r in s.admitted] == [1, 2]
    assert [r.rid for r in s.waiting] == [0]
    slow.plan_future.set_result(SimpleNamespace(out_elems=100, workspace_bytes=100))
    s._admit()
    assert [r.rid for r in s.admitted] == [1, 2, 0]


def test_oversized_request_runs_alone():
    s = _server(budget=100)
    big, small = _req(0, 1000, 1000), _req(1, 1, 256)
    s.waiting.extend([big, small])
    s._admit()
    # nothing held memory, so the oversized request is admitted; the next waits for it
    assert [r.rid for r in s.admitted] == [0]
    assert [r.rid for r in s.waiting] == [1]
    s.used -= big.nbytes
    s._admit()
    assert [r.rid for r in s.admitted] == [0, 1]


class _FakeQueue:
    def __init__(self):
        self.flags = []

    def poll(self, cap=4096):
        got, self.flags = self.flags[:cap], self.flags[cap:]
        return got


class _FakeEvent:
    def __init__(self):
        self.fired = False

    def query(self):
        return self.fired


def test_batched_workspace_stays_counted_until_the_launch_ends():
    # Requests of one persistent launch report completion one by one, but
    # their workspaces stay allocated until the launch itself has ended: the
    # budget must keep counting those bytes until then.
    s = _server(budget=10_000)
    s.keep_outputs = True
    s.finished = []
    s.queues = [_FakeQueue()]
    s.inflight = [1]
    reqs = [_req(k, 100, 600) for k in range(3)]  # 400 output + 600 workspace bytes each
    s.waiting.extend(reqs)
    s._admit()
    assert s.used == 3000
    ev = _FakeEvent()
    s.by_rid = {r.rid: r for r in reqs}
    for r in reqs:
        r.ws = object()
    s.running = [serve._Batch(ev, list(reqs), 0)]
    held = lambda: sum(r.ws_bytes for r in reqs if r.ws is not None) + sum(
        r.out_bytes for r in reqs if r.done is None)
    clock = iter(range(100))
    now = lambda: float(next(clock))
    s.queues[0].flags = [0, 1]
    s._retire(now)
    assert s.used == held() == 400 + 3 * 600
    s.queues[0].flags = [2]
    s._retire(now)
    # every request is done but the launch has not ended: workspaces still held
    assert s.used == held() == 3 * 600 and s.running and s.inflight == [1]
    ev.fired = True
    s._retire(now)
    assert s.used == held() == 0 and not s.running and s.inflight == [0]
    assert [r.rid for r in s.finished] == [0, 1, 2]


def test_native_builder_pool_host_plans():
    # The native builder pool (fht_builder_*) on host-only plans: every
    # submitted shape comes back once, equal to a plan built directly; a bad
    # size comes back as an error; unpolled plans are released by close().
    import time as _t

    import torch

    import paper_2411_07351_gb300 as F

    pool = F.PlanBuilderPool(threads=3)
    shapes = [(5, 7), (64, 65), (257, 100), (1000, 33), (4095, 17)]
    tags = {pool.submit(h, w, torch.uint8, 15, "cyclic", "T", device=-1): (h, w) for h, w in shapes}
    bad = pool.submit(0, 5, torch.uint8, 15, "cyclic", "T", device=-1)
    got, deadline = {}, _t.time() + 60
    while len(got) < len(tags) + 1 and _t.time() < deadline:
        for tag, res in pool.poll():
            got[tag] = res
        _t.sleep(0.01)
    assert sorted(got) == sorted(list(tags) + [bad])
    assert isinstance(got[bad], F.FHTError)
    for tag, (h, w) in tags.items():
        p, ref = got[tag], F.Plan(h, w, torch.uint8, 15, "cyclic", device=-1)
        assert (p.h, p.w) == (h, w)
        assert p.out_elems == ref.out_elems and p.workspace_bytes == ref.workspace_bytes
        assert p.info.model_bytes == ref.info.model_bytes and p.info.adds == ref.info.adds
    assert pool.pending() == (0, 0)
    pool.submit(300, 300, torch.uint8, 15, "extended", "T", device=-1)
    pool.close()  # finishes the queued build and destroys the unclaimed plan


class _ReadyQueue:
    def __init__(self, ready):
        self._ready = ready
        self.asked = 0

    def ready(self):
        self.asked += 1
        return self._ready


def test_batched_launch_only_on_a_queue_that_does_not_block():
    # A batched submit to a queue whose previous table copies are still queued
    # behind earlier launches would make the host wait; the loop picks the
    # least-loaded stream among those with room AND a ready queue, and launches
    # nothing this turn when there is none.  Plain launches need no queue.
    s = serve.Server.__new__(serve.Server)
    s.streams = [None] * 4
    s.max_inflight = 2
    s.inflight = [0, 1, 2, 0]
    s.queues = [_ReadyQueue(False), _ReadyQueue(True), _ReadyQueue(True), _ReadyQueue(True)]
    assert s._pick_stream(batched=False) == 0
    assert s._pick_stream(batched=True) == 3
    s.inflight = [0, 1, 2, 2]
    assert s._pick_stream(batched=True) == 1
    s.queues[1]._ready = False
    assert s._pick_stream(batched=True) is None
    assert s._pick_stream(batched=False) == 0
    assert s.queues[2].asked == 0  # a full stream's queue is not even asked


def test_lone_small_request_takes_the_per_image_kernels():
    # Small requests are batched into one persistent launch when several are
    # admitted together; one admitted alone runs the per-image kernels (three
    # short launches beat a one-job persistent launch); large ones always do.
    s = serve.Server.__new__(serve.Server)
    s.plain_pixels = 1000
    s.solo_plain = True
    small = lambda rid: serve.Request(rid=rid, arrival=0.0, image=SimpleNamespace(numel=lambda: 100))
    large = serve.Request(rid=9, arrival=0.0, image=SimpleNamespace(numel=lambda: 5000))
    s.admitted = collections.deque([small(0)])
    assert s._launch_plain()
    s.admitted = collections.deque([small(0), small(1)])
    assert not s._launch_plain()
    s.admitted = collections.deque([large, small(1)])
    assert s._launch_plain()
    s.solo_plain = False
    s.admitted = collections.deque([small(0)])
    assert not s._launch_plain()
