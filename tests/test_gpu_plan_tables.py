"""Device plans keep on the host only the tables their launches read there;
fht_plan_table and fht_plan_check copy the rest back from the device.  The
copies must equal the tables of a host-only plan of the same configuration,
before and after the lazy adjoint build, and the plans must still run."""
import ctypes

import numpy as np
import pytest
from numpy.lib.recfunctions import repack_fields
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


# tables whose elements carry a pad field (not part of the schedule): compared without it
_PADDED = {
    2: np.dtype({"names": ["top", "bot", "s", "pad"], "formats": ["<i2"] * 4}, align=True),   # MergeOp
    13: np.dtype({"names": ["top", "bot", "s", "pad"], "formats": ["<i2"] * 4}, align=True),  # MergeOp
    6: np.dtype({"names": ["dst", "q", "term_begin", "term_count", "flags", "w", "pad"],
                 "formats": ["<i8"] + ["<i4"] * 6}, align=True),                               # SpineRow
    7: np.dtype({"names": ["row", "wpart", "off", "sofs", "pad"], "formats": ["<i8"] + ["<i4"] * 4},
                align=True),                                                                    # SpineTerm
}


def _tables(F, plan):
    from paper_2411_07351_gb300 import _capi as C

    lib, out = C.load(), {}
    for k in range(14):
        data, count, esz = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int32()
        C.check(lib.fht_plan_table(plan._h, k, ctypes.byref(data), ctypes.byref(count), ctypes.byref(esz)),
                "fht_plan_table")
        n = count.value * esz.value
        raw = ctypes.string_at(data.value, n) if n else b""
        if k in _PADDED:
            dt = _PADDED[k]
            assert esz.value == dt.itemsize
            a = np.frombuffer(raw, dtype=dt)
            raw = repack_fields(a[[f for f in dt.names if f != "pad"]]).tobytes()
        out[k] = raw
    return out


@pytest.mark.parametrize("h,w,boundary,dtype", [(131, 45, "extended", torch.uint8), (300, 700, "cyclic", torch.float32),
                                                (1000, 257, "extended", torch.float32)])
def test_device_plan_tables_come_back_equal(F, h, w, boundary, dtype):
    dev = F.Plan(h, w, dtype, F.FHT_QALL, boundary)
    host = F.Plan(h, w, dtype, F.FHT_QALL, boundary, device=-1)
    x = (torch.rand(h, w, device="cuda") * 100).to(dtype)
    ref = dev.forward(x)
    assert _tables(F, dev) == _tables(F, host)
    dev.check()
    assert torch.equal(dev.forward(x), ref)
    # the lazy adjoint build replaces the tables; they are released and restored again
    out = dev.forward(x)
    gin = torch.empty((h, w), dtype=dev.out_dtype, device="cuda")
    ws = dev.new_workspace(adjoint=True)
    dev.adjoint(out, gin, ws)
    host_adj = F.Plan(h, w, dtype, F.FHT_QALL, boundary, device=-1, with_adjoint=True)
    assert _tables(F, dev) == _tables(F, host_adj)
    dev.check()
    gin2 = torch.empty_like(gin)
    dev.adjoint(out, gin2, ws)
    assert torch.equal(gin, gin2)


def test_table_ranges_reused_after_destroy(F, orc):
    # Plans take their device tables from ranges of shared chunks; a destroyed
    # plan's range goes to later plans.  Many plans built and destroyed in an
    # interleaved order, then every surviving plan (old ones and ones on
    # recycled ranges, small and large) still
    # gives the oracle's transform bit for bit.
    rng = np.random.default_rng(17)
    shapes = [(int(rng.integers(1, 90)), int(rng.integers(1, 90))) for _ in range(300)]
    shapes += [(2000, 1900), (1500, 64)]
    plans = {k: F.Plan(h, w, torch.uint8, 15, "cyclic") for k, (h, w) in enumerate(shapes)}
    for k in list(plans)[::2]:
        plans.pop(k).close()
    more = [(int(rng.integers(1, 90)), int(rng.integers(1, 90))) for _ in range(150)]
    for j, (h, w) in enumerate(more):
        plans[len(shapes) + j] = F.Plan(h, w, torch.uint8, 15, "extended")
    shapes += more
    for k in sorted(plans)[::7] + [len(shapes) - len(more) - 1]:
        p = plans[k]
        img = rng.integers(0, 256, size=(p.h, p.w)).astype(np.uint8)
        got = p.forward(torch.from_numpy(img).cuda()).cpu().numpy().astype(np.int64)
        b = orc.EXTENDED if p.boundary == "extended" else orc.CYCLIC
        ref = orc.fht(img.astype(np.int64), 15, b, orc.SPLIT_T)
        assert np.array_equal(got, ref), (k, p.h, p.w, p.boundary)
