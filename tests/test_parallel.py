"""Multi-GPU host logic on CPU: sharding of independent images across ranks
and the max / sum over ranks, run as two gloo processes."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2411_07351_gb300.parallel import cost, gather_by_index, max_over_ranks, my_shard, route, shard, sum_over_ranks


def test_shard_covers_every_image_once_and_balances():
    import numpy as np

    g = np.random.default_rng(0)
    sizes = [tuple(int(v) for v in g.integers(17, 512, 2)) for _ in range(500)]
    for world in (1, 2, 3, 8):
        parts = shard(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(cost(*sizes[i]) for i in p) for p in parts]
        assert max(loads) <= 1.02 * (sum(loads) / world) + max(cost(*s) for s in sizes)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = shard(sizes, world)
    mine = parts[rank]
    # each rank "processes" its images: pixels as the unit of work
    pix = float(sum(sizes[i][0] * sizes[i][1] for i in mine))
    total = sum_over_ranks(pix)
    slow = max_over_ranks(float(rank + 1))
    q.put((rank, mine, total, slow))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    sizes = [(17 + 13 * k, 300 - 7 * k) for k in range(30)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    all_idx = sorted(res[0][1] + res[1][1])
    assert all_idx == list(range(len(sizes)))
    want = float(sum(h * w for h, w in sizes))
    assert res[0][2] == want and res[1][2] == want
    assert res[0][3] == 2.0 and res[1][3] == 2.0


def test_route_balances_a_stream_identically():
    import numpy as np

    g = np.random.default_rng(2)
    sizes = [tuple(int(v) for v in g.integers(64, 4097, 2)) for _ in range(2000)]
    for world in (1, 2, 4):
        r1, r2 = route(sizes, world), route(list(sizes), world)
        assert r1 == r2 and set(r1) <= set(range(world))
        loads = [sum(cost(*sizes[i]) for i in range(len(sizes)) if r1[i] == k) for k in range(world)]
        assert max(loads) - min(loads) <= max(cost(*s) for s in sizes)


def _transform_worker(rank, world, port, seed, q):
    # each rank transforms its shard of a seeded batch (the oracle stands in
    # for the device here: this checks the sharding and the gather, on CPU)
    import numpy as np

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = np.random.default_rng(seed)
    imgs = [g.integers(0, 256, size=tuple(int(v) for v in g.integers(1, 40, 2)), dtype=np.uint8) for _ in range(25)]
    mine = my_shard([im.shape for im in imgs])
    local = {i: oracle.fht(imgs[i].astype(np.int64), 15, oracle.CYCLIC) for i in mine}
    merged = gather_by_index(local)
    q.put((rank, sorted(mine), {k: v.tolist() for k, v in merged.items()} if rank == 0 else None))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_transforms_equal_single_rank(orc):
    import numpy as np

    seed = 9
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_transform_worker, args=(r, 2, port, seed, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(res[0][1] + res[1][1]) == list(range(25)) and not set(res[0][1]) & set(res[1][1])
    merged = res[0][2]
    g = np.random.default_rng(seed)
    imgs = [g.integers(0, 256, size=tuple(int(v) for v in g.integers(1, 40, 2)), dtype=np.uint8) for _ in range(25)]
    assert sorted(merged) == list(range(25))
    for i, im in enumerate(imgs):
        assert merged[i] == orc.fht(im.astype(np.int64), 15, orc.CYCLIC).tolist()
