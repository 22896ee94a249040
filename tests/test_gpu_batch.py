"""Batched persistent launch (fht_submit) against per-image fht_forward and
the oracle: bit-exact for integer images, alone and in the mix, in any order."""
import numpy as np
import pytest
import torch

from paper_2411_07351_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_07351_gb300 import build as B

    B.build()
    import paper_2411_07351_gb300 as F

    return F


@pytest.fixture(scope="module")
def queue(F):
    from paper_2411_07351_gb300.batch import BatchQueue

    q = BatchQueue(max_jobs=512, max_units=1 << 20)
    yield q
    q.close()


def _edge_maps(seed, count, lo=17, hi=511):
    imgs = inputs.c3_batch(seed=seed, count=count, lo=lo, hi=hi)
    return [torch.from_numpy(im).cuda() for im in imgs]


def test_batch_matches_single_and_oracle(F, orc, queue):
    xs = _edge_maps(3, 96)
    outs, plans, _ = queue.submit(xs, 15, "cyclic")
    torch.cuda.synchronize()
    assert queue.status() == 0
    for x, o, p in zip(xs, outs, plans):
        ref = p.forward(x)
        assert torch.equal(o, ref)
    for k in (0, 5, 50):
        im = xs[k].cpu().numpy().astype(np.int64)
        assert np.array_equal(outs[k].cpu().numpy(), orc.fht(im, 15, orc.CYCLIC))


@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_batch_mixed_sizes_and_order(F, queue, boundary):
    # tiny (fused only), 64 < n (spine), powers of two (band root), larger bands
    g = np.random.default_rng(7)
    sizes = [(17, 30), (64, 64), (65, 17), (128, 40), (200, 511), (511, 200), (256, 256), (1, 9), (300, 1)]
    xs = [torch.from_numpy(g.integers(0, 256, s, dtype=np.uint8)).cuda() for s in sizes]
    outs, plans, _ = queue.submit(xs, 15, boundary)
    torch.cuda.synchronize()
    assert queue.status() == 0
    ref = [p.forward(x) for x, p in zip(xs, plans)]
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    order = list(range(len(xs)))[::-1]
    outs2, _, _ = queue.submit([xs[i] for i in order], 15, boundary)
    torch.cuda.synchronize()
    for k, i in enumerate(order):
        assert torch.equal(outs2[k], ref[i])


@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_batch_chunked_spines_and_tall_roots(F, orc, queue, boundary):
    # spines of several chunks (one phase per chunk in the persistent launch)
    # and a root taller than 8192 rows (its big part summed first)
    g = np.random.default_rng(11)
    sizes = [(2047, 50), (50, 2047), (1500, 33), (9000, 3), (3, 9000), (700, 700)]
    xs = [torch.from_numpy(g.integers(0, 256, s, dtype=np.uint8)).cuda() for s in sizes]
    outs, plans, _ = queue.submit(xs, 15, boundary)
    torch.cuda.synchronize()
    assert queue.status() == 0
    for x, o, p in zip(xs, outs, plans):
        assert torch.equal(o, p.forward(x))
    b = orc.EXTENDED if boundary == "extended" else orc.CYCLIC
    for k in (0, 3):
        im = xs[k].cpu().numpy().astype(np.int64)
        assert np.array_equal(outs[k].cpu().numpy(), orc.fht(im, 15, b))


def test_batch_float_and_split_s(F, queue):
    g = np.random.default_rng(8)
    xs = [torch.from_numpy(g.standard_normal(s).astype(np.float32)).cuda() for s in [(70, 90), (300, 129), (33, 500)]]
    outs, plans, _ = queue.submit(xs, 15, "extended", "S")
    torch.cuda.synchronize()
    assert queue.status() == 0
    for x, o, p in zip(xs, outs, plans):
        assert torch.equal(o, p.forward(x))


def test_batch_withheld_dependency_times_out(F):
    """The bounded wait: a job whose later units wait for a unit that never
    exists makes the kernel record FHT_ERR_TIMEOUT and return; the context
    stays usable."""
    from paper_2411_07351_gb300 import _capi
    from paper_2411_07351_gb300.batch import BatchQueue

    q = BatchQueue(max_jobs=8, max_units=1 << 16)
    q.set_wait_limit(0.05)
    xs = _edge_maps(5, 3, lo=100, hi=300)
    q.submit(xs, 15, "cyclic", flags=[0, _capi.FHT_JOB_WITHHOLD_DEPENDENCY, 0])
    torch.cuda.synchronize()
    assert q.status() == _capi.FHT_ERR_TIMEOUT
    q.reset_status()
    outs, plans, _ = q.submit(xs, 15, "cyclic")
    torch.cuda.synchronize()
    assert q.status() == 0
    for x, o, p in zip(xs, outs, plans):
        assert torch.equal(o, p.forward(x))
    q.close()


def test_batch_poll_tags(F, queue):
    torch.cuda.synchronize()
    queue.poll(1 << 16)  # drain the tags of earlier submits
    xs = _edge_maps(9, 4)
    queue.submit(xs, 15, "cyclic", tags=[11, 12, 13, 14])
    torch.cuda.synchronize()
    assert sorted(queue.poll()) == [11, 12, 13, 14]
    assert queue.poll() == []
    # jobs are reported one by one: after a submit finishes, polling with a
    # small cap returns the tags in pieces
    queue.submit(xs, 15, "cyclic", tags=[21, 22, 23, 24])
    torch.cuda.synchronize()
    got = queue.poll(cap=3) + queue.poll(cap=3)
    assert sorted(got) == [21, 22, 23, 24]


def test_queue_ready_tracks_the_staging_copies(F, queue):
    # fht_queue_ready: 0 while a submit's table copies wait behind earlier
    # work on the stream, 1 once they have run; a submit to a ready queue
    # does not wait on the host
    torch.cuda.synchronize()
    assert queue.ready()
    s = torch.cuda.Stream()
    xs = _edge_maps(5, 3)
    with torch.cuda.stream(s):
        torch.cuda._sleep(50_000_000)  # tens of milliseconds of device work ahead of the copies
        queue.submit(xs, 15, "cyclic", stream=s)
    assert not queue.ready()
    s.synchronize()
    assert queue.ready()
    with torch.cuda.stream(s):
        outs, plans, _ = queue.submit(xs, 15, "cyclic", stream=s)
    s.synchronize()
    for x, o, p in zip(xs, outs, plans):
        assert torch.equal(o, p.forward(x))


def test_batch_graph_replay(F, queue):
    """A fixed batch captured in a CUDA graph replays to the same results."""
    xs = _edge_maps(10, 16)
    outs, plans, ws = queue.submit(xs, 15, "cyclic")
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        for o in outs:
            o.zero_()
        with torch.cuda.graph(graph, stream=s, capture_error_mode="relaxed"):
            queue.submit(xs, 15, "cyclic", outs=outs, workspaces=ws, stream=s)
    torch.cuda.synchronize()
    for o in outs:
        o.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)


def test_batch_c3_full_size(F, orc):
    """The full batching workload (4096 binary edge maps, h, w ~ U{17..511}, all
    four quadrants, cyclic) in one persistent launch: every output equals the
    oracle bit for bit (the oracle spread over the host's cores, compared by
    digest, any differing image recomputed), and the per-image launches too."""
    from oracle import parallel
    from paper_2411_07351_gb300.batch import BatchQueue

    imgs = inputs.c3_batch()
    want = parallel.int32_digests(imgs, 15, orc.CYCLIC)
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    q = BatchQueue(max_jobs=len(xs), max_units=1 << 23)
    outs, plans, _ = q.submit(xs, 15, "cyclic")
    torch.cuda.synchronize()
    assert q.status() == 0
    bad = [k for k, o in enumerate(outs) if parallel.digest(o.cpu().numpy()) != want[k]]
    for k in bad[:3]:
        ref = orc.fht(imgs[k].astype(np.int64), 15, orc.CYCLIC)
        got = outs[k].cpu().numpy()
        i = int(np.argmax(got != ref))
        pytest.fail(f"image {k} ({imgs[k].shape}): first difference at packed index {i}: {got[i]} vs {ref[i]}")
    assert not bad
    for x, o, p in zip(xs, outs, plans):
        assert torch.equal(o, p.forward(x))
    q.close()


def test_batch_register_tiled_plans(F, orc):
    """Plans with the register-tiled launch shape (tile 192, 256 threads,
    32-column generic tiles) submitted to the batched launch: its 64-row block
    and band units take the register-tiled path, bit-exact against the oracle."""
    from paper_2411_07351_gb300.batch import BatchQueue

    g = np.random.default_rng(17)
    sizes = [(64, 300), (200, 511), (300, 90), (511, 200), (1100, 40), (65, 17)]
    imgs = [g.integers(0, 256, s, dtype=np.uint8) for s in sizes]
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    q = BatchQueue(max_jobs=16, max_units=1 << 18)
    for boundary in ("cyclic", "extended"):
        plans = [F.Plan(h, w, torch.uint8, 15, boundary, tile_cols=192, threads=256, generic_cols=32)
                 for h, w in sizes]
        outs, _, _ = q.submit(xs, 15, boundary, plans=plans)
        torch.cuda.synchronize()
        assert q.status() == 0
        b = orc.EXTENDED if boundary == "extended" else orc.CYCLIC
        for im, o in zip(imgs, outs):
            assert np.array_equal(o.cpu().numpy(), orc.fht(im.astype(np.int64), 15, b))
    q.close()


def test_batch_tuner_picks_a_measured_shape(F, orc):
    """tune.tune_batch times every candidate plan shape on the batch itself
    and returns the fastest; a queue with that shape gives the oracle's result."""
    from paper_2411_07351_gb300 import tune
    from paper_2411_07351_gb300.batch import BatchQueue

    imgs = inputs.c3_batch(seed=5, count=24)
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    best = tune.tune_batch(xs, 15, "cyclic", "T", reps=2)
    assert best["shape"] in [tuple(c) for c in tune.BATCH_CANDIDATES]
    assert best["ms"] == min(c[1] for c in best["candidates"])
    q = BatchQueue(max_jobs=len(xs), shape=best["shape"])
    outs, _, _ = q.submit(xs, 15, "cyclic")
    torch.cuda.synchronize()
    for im, o in zip(imgs, outs):
        assert np.array_equal(o.cpu().numpy(), orc.fht(im.astype(np.int64), 15, orc.CYCLIC))
    q.close()
