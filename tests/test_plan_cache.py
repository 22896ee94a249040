"""The LRU plan cache that the batch queue and the server share (CPU only,
host-only plans)."""
import concurrent.futures as cf

import pytest
import torch


@pytest.fixture(scope="module")
def F():
    from paper_2411_07351_gb300 import build as B

    B.build()
    import paper_2411_07351_gb300 as F

    return F


def _get(cache, h, w, tile_cols=0):
    return cache.get(h, w, torch.uint8, 15, "cyclic", "T", -1, tile_cols=tile_cols)


def test_hits_return_the_same_plan_and_lru_evicts(F):
    from paper_2411_07351_gb300.fht import PlanCache

    c = PlanCache(capacity=2)
    a, b = _get(c, 10, 20), _get(c, 30, 40)
    assert _get(c, 10, 20) is a  # hit; a becomes the most recent
    d = _get(c, 50, 60)          # evicts b, the least recently used
    assert _get(c, 10, 20) is a and _get(c, 50, 60) is d
    b2 = _get(c, 30, 40)
    assert b2 is not b and (b2.h, b2.w) == (30, 40)
    # evicted plans are dropped, not closed: a caller still holding one can use it
    assert b.info.out_elems == b2.info.out_elems


def test_every_configuration_field_is_part_of_the_key(F):
    from paper_2411_07351_gb300.fht import PlanCache

    c = PlanCache(capacity=16)
    base = _get(c, 64, 64)
    assert _get(c, 64, 64, tile_cols=64) is not base
    assert c.get(64, 64, torch.float32, 15, "cyclic", "T", -1) is not base
    assert c.get(64, 64, torch.uint8, 1, "cyclic", "T", -1) is not base
    assert c.get(64, 64, torch.uint8, 15, "extended", "T", -1) is not base
    assert c.get(64, 64, torch.uint8, 15, "cyclic", "S", -1) is not base
    assert _get(c, 64, 64) is base


def test_concurrent_gets_return_usable_plans(F):
    from paper_2411_07351_gb300.fht import PlanCache

    c = PlanCache(capacity=4)
    shapes = [(17 + k % 6, 33 + k % 5) for k in range(48)]
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        plans = list(ex.map(lambda s: _get(c, *s), shapes))
    for (h, w), p in zip(shapes, plans):
        assert (p.h, p.w) == (h, w)
        p.check()
    assert len(c._d) <= 4
