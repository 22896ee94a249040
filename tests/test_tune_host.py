"""Host side of the autotuner (CPU only): buckets, cache precedence and the
packaged table.  Timing needs a GPU (tests/test_gpu_tune.py); here every
packaged choice is checked to be a candidate whose plan passes the host
verifier, so a table entry can never select a launch shape the kernels do
not support.
"""
import json

import pytest
import torch

from paper_2411_07351_gb300 import tune


@pytest.fixture(scope="module")
def F():
    from paper_2411_07351_gb300 import build as B

    B.build()
    import paper_2411_07351_gb300 as F

    return F


def test_bucket_is_a_half_octave_grid():
    assert [tune.bucket(n) for n in (64, 91, 128, 181, 256, 4096)] == [64, 91, 128, 181, 256, 4096]
    # neighbours of a grid point fall into it
    assert tune.bucket(100) == 91 and tune.bucket(120) == 128 and tune.bucket(4095) == 4096
    assert tune.bucket(0) == 1 and tune.bucket(1) == 1


def test_key_names_every_field():
    assert tune.key(4095, 300, torch.float32, 15, "extended", "T") == "4096x256:float32:q15:extended:T"
    assert tune.key(64, 64, torch.uint8, 1, "cyclic", "S") == "64x64:uint8:q1:cyclic:S"


def test_user_cache_wins_over_packaged_table(tmp_path, monkeypatch):
    monkeypatch.setenv("FHT_TUNE_CACHE", str(tmp_path / "t.json"))
    k = tune.key(1024, 1024, torch.float32, 15, "cyclic", "T")
    packaged = tune.lookup(1024, 1024, torch.float32, 15, "cyclic", "T")
    assert packaged is not None  # shipped with the package
    tune.save_cache({k: {"tile_cols": 64, "threads": 256, "fused_rows": 64, "ms": 1.0}})
    hit = tune.lookup(1024, 1024, torch.float32, 15, "cyclic", "T")
    assert hit["tile_cols"] == 64 and hit["threads"] == 256


def test_corrupt_cache_falls_back_to_packaged(tmp_path, monkeypatch):
    p = tmp_path / "t.json"
    p.write_text("{not json")
    monkeypatch.setenv("FHT_TUNE_CACHE", str(p))
    assert tune.load_cache() == {}
    assert tune.lookup(1024, 1024, torch.float32, 15, "cyclic", "T") is not None


def _packaged():
    with open(tune.PACKAGED) as f:
        return json.load(f)


def test_packaged_entries_are_candidates():
    table = _packaged()
    assert len(table) >= 40
    for k, v in table.items():
        assert (v["tile_cols"], v["threads"], v["fused_rows"]) in tune.CANDIDATES, k
        # the kept choice is the fastest candidate measured
        assert v["ms"] == min(c[3] for c in v["candidates"]), k
        assert len(v["candidates"]) == len(tune.CANDIDATES), k


@pytest.mark.parametrize("entry", sorted(_packaged())[::4])
def test_packaged_choice_builds_a_verified_plan(F, entry):
    v = _packaged()[entry]
    hb, wb = (int(x) for x in entry.split(":")[0].split("x"))
    dtype = {"float32": torch.float32, "uint8": torch.uint8}[entry.split(":")[1]]
    quads = int(entry.split(":")[2][1:])
    boundary, split = entry.split(":")[3], entry.split(":")[4]
    for h, w in ((hb, wb), (hb - 1, wb + 3)):
        p = F.Plan(h, w, dtype, quads, boundary, split=split, tile_cols=v["tile_cols"], threads=v["threads"],
                   fused_rows=v["fused_rows"], device=-1)
        p.check()
