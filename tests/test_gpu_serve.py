"""Serving loop with continuous batching: every served result equals the
oracle (bit-exact, uint8 -> int32) and the same image transformed alone;
sizes span the serving workload's log-uniform range [64, 4096], so both the
batched launches and the per-image kernels of large requests serve; admission
never exceeds the memory budget (except a lone oversize request)."""
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
    """Requests whose images are windows of one seeded uint8 field with 10 %
    non-zero pixels; returns the requests and the host copies of their images."""
    from paper_2411_07351_gb300.serve import Request

    g = np.random.Generator(np.random.PCG64(seed))
    field_np = np.where(g.random((hi, hi)) < 0.1, g.integers(1, 256, (hi, hi)), 0).astype(np.uint8)
    field = torch.from_numpy(field_np).cuda()
    t, reqs, host = 0.0, [], []
    for k in range(n):
        t += g.exponential(1.0 / rate)
        h = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        w = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        y0, x0 = int(g.integers(0, hi - h + 1)), int(g.integers(0, hi - w + 1))
        reqs.append(Request(k, t, field[y0:y0 + h, x0:x0 + w]))
        host.append(field_np[y0:y0 + h, x0:x0 + w])
    return reqs, host


def _check_against_oracle(done, host):
    from oracle import parallel

    want = parallel.int32_digests(host, 15, 0)
    bad = [r.rid for r in done if parallel.digest(r.out.cpu().numpy()) != want[r.rid]]
    assert not bad, f"served outputs differing from the oracle: {bad[:10]}"


def test_served_results_equal_oracle_and_single(F):
    from paper_2411_07351_gb300.serve import Server, run_stream

    reqs, host = _requests(300, 4000.0, 64, 700, 6)
    # solo_plain off: every small request goes through the persistent batch launch
    srv = Server(budget_bytes=1 << 30, streams=3, solo_plain=False)
    done, wall = run_stream(srv, reqs)
    assert len(done) == len(reqs)
    assert srv.max_used <= 1 << 30
    assert max(r.batch_size for r in done) > 1  # requests really were batched together
    _check_against_oracle(done, host)
    for r in done:
        ref = r.plan.forward(r.image)
        assert torch.equal(r.out, ref), r.rid
    srv.close()


def test_served_full_size_range(F):
    """The serving workload's size range, log-uniform in [64, 4096] for h and w
    independently, at 2000 requests per second under the 16 GB budget."""
    from paper_2411_07351_gb300.serve import Server, run_stream

    reqs, host = _requests(48, 2000.0, 64, 4096, 61)
    srv = Server(budget_bytes=16 << 30, solo_plain=False)
    done, _ = run_stream(srv, reqs)
    assert len(done) == len(reqs)
    assert srv.max_used <= 16 << 30
    big = [r for r in done if r.image.numel() >= srv.plain_pixels]
    small = [r for r in done if r.image.numel() < srv.plain_pixels]
    assert big and small  # both the per-image kernels and the batched launches served
    assert max(r.batch_size for r in small) > 1
    _check_against_oracle(done, host)
    for r in done:
        assert torch.equal(r.out, r.plan.forward(r.image)), r.rid
    srv.close()


def test_served_default_policy_equals_oracle(F):
    """The default policy at a low arrival rate: most small requests arrive
    alone and take the per-image kernels, any that meet in one turn share a
    persistent launch; every output equals the oracle's."""
    from paper_2411_07351_gb300.serve import Server, run_stream

    reqs, host = _requests(60, 500.0, 64, 1500, 8)
    srv = Server(budget_bytes=4 << 30)
    done, _ = run_stream(srv, reqs)
    assert len(done) == len(reqs)
    _check_against_oracle(done, host)
    srv.close()


def test_admission_budget_smaller_than_a_request(F):
    from paper_2411_07351_gb300.serve import Server, run_stream

    reqs, _ = _requests(20, 2000.0, 200, 400, 7)
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

    reqs, host = _requests(50, 2000.0, 64, 300, 8)
    srv = PlainServer()
    done, _ = run_stream(srv, reqs)
    assert len(done) == 50
    _check_against_oracle(done, host)
    for r in done:
        assert torch.equal(r.out, r.plan.forward(r.image))
