"""Serving loop with continuous batching: every result equals the plain
single-image transform (bit-exact, uint8 -> int32), alone and in the mix;
admission never exceeds the memory budget (except a lone oversize request)."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_07351_gb300 import build as B

    B.build()
    import paper_2411_07351_gb300 as F

    return F


def _requests(n, rate, lo, hi, seed):
    from paper_2411_07351_gb300.serve import Request

    g = np.random.Generator(np.random.PCG64(seed))
    field = torch.from_numpy(np.where(g.random((hi, hi)) < 0.1, g.integers(1, 256, (hi, hi)), 0)
                             .astype(np.uint8)).cuda()
    t, reqs = 0.0, []
    for k in range(n):
        t += g.exponential(1.0 / rate)
        h = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        w = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        y0, x0 = int(g.integers(0, hi - h + 1)), int(g.integers(0, hi - w + 1))
        reqs.append(Request(k, t, field[y0:y0 + h, x0:x0 + w]))
    return reqs


def test_served_results_equal_single(F):
    from paper_2411_07351_gb300.serve import Server, run_stream

    reqs = _requests(300, 4000.0, 64, 700, 6)
    srv = Server(budget_bytes=1 << 30, streams=3)
    done, wall = run_stream(srv, reqs)
    assert len(done) == len(reqs)
    assert srv.max_used <= 1 << 30
    assert max(r.batch_size for r in done) > 1  # requests really were batched together
    for r in done:
        ref = r.plan.forward(r.image)
        assert torch.equal(r.out, ref), r.rid
    srv.close()


def test_admission_budget_smaller_than_a_request(F):
    from paper_2411_07351_gb300.serve import Server, run_stream

    reqs = _requests(20, 2000.0, 200, 400, 7)
    srv = Server(budget_bytes=1 << 20, streams=2)  # 1 MiB: every request alone exceeds it
    done, _ = run_stream(srv, reqs)
    assert len(done) == 20
    assert max(r.batch_size for r in done) == 1  # admitted one at a time
    assert srv.max_used <= max(r.nbytes for r in done)
    for r in done:
        assert torch.equal(r.out, r.plan.forward(r.image))
    srv.close()


def test_plain_server(F):
    from paper_2411_07351_gb300.serve import PlainServer, run_stream

    reqs = _requests(50, 2000.0, 64, 300, 8)
    srv = PlainServer()
    done, _ = run_stream(srv, reqs)
    assert len(done) == 50
    for r in done:
        assert torch.equal(r.out, r.plan.forward(r.image))
