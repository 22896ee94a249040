"""Host-side tests of libfht.so: exports, host-only plans, the byte/addition
model and the plan verifier.  No GPU is touched."""
import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_2411_07351_gb300 import build as B

    B.build()
    import paper_2411_07351_gb300 as F

    return F


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fht_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(F):
    from paper_2411_07351_gb300 import _capi

    lib = ctypes.CDLL(_capi.LIB_PATH)
    declared = _declared_functions()
    assert {"fht_plan", "fht_forward", "fht_adjoint", "fht_plan_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(_capi.SIGNATURES) <= declared | set()


def test_status_strings(F):
    from paper_2411_07351_gb300 import _capi

    lib = _capi.load()
    assert lib.fht_status_string(0) == b"FHT_OK"
    assert lib.fht_status_string(4) == b"FHT_ERR_TIMEOUT"


@pytest.mark.parametrize("n", [2, 3, 17, 257, 1000, 4095])
def test_adds_match_theorem1(F, orc, n):
    # cyclic, one quadrant of an n x n image: the plan's count is f_T(n) (Theorem 1)
    p = F.Plan(n, n, torch.float32, 1, "cyclic", "T", device=-1)
    assert p.info.adds == orc.adds(n, orc.SPLIT_T)
    p = F.Plan(n, n, torch.float32, 1, "cyclic", "S", device=-1)
    assert p.info.adds == orc.adds(n, orc.SPLIT_S)


def test_shapes_and_offsets(F, orc):
    for h, w, b in [(13, 11, "extended"), (4095, 4095, "extended"), (1, 7, "cyclic")]:
        p = F.Plan(h, w, torch.float32, 15, b, device=-1)
        ob = orc.EXTENDED if b == "extended" else orc.CYCLIC
        assert p.shapes == orc.out_shape(h, w, 15, ob)
        assert p.out_elems == orc.out_elems(h, w, 15, ob)


def test_plan_verifier_over_many_shapes(F):
    sizes = list(range(1, 40)) + [63, 64, 65, 127, 129, 255, 257, 511, 513, 896, 4095, 4097]
    for h in sizes:
        for w in (1, 2, 5, 33, 64, 100):
            for b in ("cyclic", "extended"):
                for sp in ("T", "S"):
                    F.Plan(h, w, torch.uint8, 15, b, sp, device=-1, with_adjoint=(h + w) % 3 == 0).check()
    for fr in (1, 2, 8, 32, 64):
        for tc in (32, 96, 256):
            F.Plan(300, 77, torch.float64, 15, "extended", device=-1, fused_rows=fr, tile_cols=tc,
                   with_adjoint=True).check()


def test_plan_verifier_spine_chunks_and_tall_roots(F):
    # spine chunk sizes, and roots taller than 8192 rows (their power-of-two
    # part is summed from 4096-row bands before the spine)
    for h in (2047, 4095, 8191, 8193, 9000, 16384, 20000, 40000):
        for ch in (1, 2, 3, 100):
            for b in ("cyclic", "extended"):
                F.Plan(h, 3, torch.float32, 15, b, device=-1, spine_chunk=ch).check()
    with pytest.raises(F.FHTError):
        F.Plan(100, 100, torch.float32, 15, device=-1, spine_chunk=-1)


def test_invalid_arguments(F):
    with pytest.raises(F.FHTError):
        F.Plan(0, 5, torch.float32, 1, device=-1)
    with pytest.raises(F.FHTError):
        F.Plan(5, 70000, torch.float32, 1, device=-1)
    with pytest.raises(F.FHTError):
        F.Plan(5, 5, torch.float32, 0, device=-1)
    with pytest.raises(F.FHTError):
        F.Plan(5, 5, torch.float32, 1, device=-1, fused_rows=48)


def test_host_only_plan_cannot_run(F):
    from paper_2411_07351_gb300 import _capi

    p = F.Plan(8, 8, torch.float32, 1, device=-1)
    lib = _capi.load()
    st = lib.fht_forward(p._h, 16, 8, 16, 256, p.workspace_bytes, None)
    assert st == _capi.FHT_ERR_INVALID
    assert b"host-only" in lib.fht_last_error()


def test_argument_errors_without_a_gpu(F):
    # every entry point checks its arguments before touching a device
    from paper_2411_07351_gb300 import _capi

    lib = _capi.load()
    p = F.Plan(8, 8, torch.float32, 1, device=-1)
    h = ctypes.c_void_p()
    assert lib.fht_pipe_create(ctypes.byref(h), p._h, 2, 1) == _capi.FHT_ERR_INVALID
    assert b"host-only" in lib.fht_last_error()
    assert lib.fht_pipe_create(ctypes.byref(h), None, 2, 1) == _capi.FHT_ERR_INVALID
    assert lib.fht_pipe_submit(None, 16, 8, 16) == _capi.FHT_ERR_INVALID
    assert lib.fht_pipe_sync(None) == _capi.FHT_ERR_INVALID
    assert lib.fht_pipe_destroy(None) == _capi.FHT_OK
    assert lib.fht_forward_noalloc(p._h, 16, 8, 16, None) == _capi.FHT_ERR_INVALID
    assert lib.fht_submit(None, 1, None, None) == _capi.FHT_ERR_INVALID
    assert lib.fht_queue_destroy(None) == _capi.FHT_OK
    r = ctypes.c_int32(7)
    assert lib.fht_queue_ready(None, ctypes.byref(r)) == _capi.FHT_ERR_INVALID
    assert lib.fht_queue_ready(None, None) == _capi.FHT_ERR_INVALID
    bp = ctypes.c_void_p()
    assert lib.fht_builder_create(ctypes.byref(bp), 0) == _capi.FHT_ERR_INVALID
    assert lib.fht_builder_poll(None, None, None, None, 0, None) == _capi.FHT_ERR_INVALID
    assert lib.fht_builder_destroy(None) == _capi.FHT_OK
    assert lib.fht_adjoint(p._h, 16, 16, 8, 256, p.adjoint_workspace_bytes, None) == _capi.FHT_ERR_INVALID
    assert lib.fht_pattern_errors(0, 5, 0, None, None) == _capi.FHT_ERR_INVALID
    assert lib.fht_plan_check(None) == _capi.FHT_ERR_INVALID
    assert lib.fht_plan_destroy(None) == _capi.FHT_OK


def test_byte_model_c2(F):
    # 4095^2 float32, four quadrants, extended; ideal = input once + output once.
    # Band schedule (Split_T, 64-row blocks): fused pass + band pass + spine sum,
    # 2.05 GB in one spine launch; summing the spine in chunks of three nodes
    # (the default) writes and reads the 511-row inner node once more: + 75 MB.
    # The per-height schedule (here forced by 32-row fused subtrees) moves one
    # read + write of every node per tree height: 5.1 GB.
    p = F.Plan(4095, 4095, torch.float32, 15, "extended", device=-1)
    assert abs(p.info.ideal_bytes - (4 * 4095 * 4095 * 4 + 4 * 4095 * 8189 * 4)) == 0
    assert 2.1e9 < p.info.model_bytes < 2.15e9
    p1 = F.Plan(4095, 4095, torch.float32, 15, "extended", device=-1, spine_chunk=100)
    assert 2.0e9 < p1.info.model_bytes < 2.1e9
    inner = 4 * 2 * 511 * (4095 + 510) * 4
    assert abs(p.info.model_bytes - p1.info.model_bytes - inner) < 1e6
    assert p.info.upper_passes == 6
    p32 = F.Plan(4095, 4095, torch.float32, 15, "extended", device=-1, fused_rows=32)
    assert 5.0e9 < p32.info.model_bytes < 5.2e9
