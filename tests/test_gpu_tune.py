"""Autotuner: every candidate launch shape gives the same (bit-exact) result;
the winner is cached and picked up by Plan(..., tuning="auto")."""
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


def test_candidates_agree_and_cache(F, tmp_path, monkeypatch):
    from paper_2411_07351_gb300 import tune

    monkeypatch.setenv("FHT_TUNE_CACHE", str(tmp_path / "tune.json"))
    g = np.random.default_rng(1)
    img = torch.from_numpy(g.integers(0, 256, (300, 200), dtype=np.uint8)).cuda()
    ref = None
    for tc, th, fr in tune.CANDIDATES:
        p = F.Plan(300, 200, torch.uint8, 15, "extended", tile_cols=tc, threads=th, fused_rows=fr)
        p.check()
        out = p.forward(img)
        if ref is None:
            ref = out.clone()
        assert torch.equal(out, ref), (tc, th, fr)
    best = tune.tune(300, 200, torch.uint8, 15, "extended", "T", reps=3)
    assert (best["tile_cols"], best["threads"], best["fused_rows"]) in [tuple(c) for c in tune.CANDIDATES]
    p = F.Plan(300, 200, torch.uint8, 15, "extended", tuning="auto")
    assert p.info.tile_cols == best["tile_cols"] and p.info.fused_rows == best["fused_rows"]
    assert torch.equal(p.forward(img), ref)
