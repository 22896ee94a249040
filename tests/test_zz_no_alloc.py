"""fht_forward_noalloc: the forward transform for callers that cannot allocate
device memory when they run it (its workspace is a fixed array inside
libfht.so).  Checked through the C ABI against fht_forward, on two calls in a
row that share the array.  Kept in its own file so that it runs last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2411_07351_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_07351_gb300 import _capi
    from paper_2411_07351_gb300 import build as B

    B.build()
    return _capi.load()


def _plan(h, w, dtype, boundary):
    import paper_2411_07351_gb300 as F

    return F.Plan(h, w, dtype, F.FHT_QALL, boundary)


def _both(lib, plan, x):
    from paper_2411_07351_gb300 import _capi

    s = torch.cuda.current_stream().cuda_stream
    ref = plan.forward(x)
    got = torch.full_like(ref, -7)
    _capi.check(lib.fht_forward_noalloc(plan._h, x.data_ptr(), x.stride(0), got.data_ptr(), s),
                "fht_forward_noalloc")
    torch.cuda.synchronize()
    return ref, got


def test_noalloc_matches_forward_twice(lib):
    # u8 -> int32: bit-exact, as for every integer path
    a = torch.from_numpy(inputs.uniform_u8(21, 257, 190)).cuda()
    b = torch.from_numpy(inputs.uniform_u8(22, 300, 301)).cuda()
    for x, boundary in ((a, "extended"), (b, "cyclic")):
        ref, got = _both(lib, _plan(x.shape[0], x.shape[1], torch.uint8, boundary), x)
        assert torch.equal(ref, got)
    # float32: within 1e-5 of the pattern L1 mass, the float tolerance of the tests
    c = torch.from_numpy(inputs.normal_f32(23, 500, 333)).cuda()
    d = torch.from_numpy(inputs.normal_f32(24, 129, 700)).cuda()
    for x in (c, d):
        p = _plan(x.shape[0], x.shape[1], torch.float32, "extended")
        ref, got = _both(lib, p, x)
        mass = p.forward(x.abs())
        torch.cuda.synchronize()
        assert bool(((ref - got).abs() <= 1e-5 * mass).all())


def test_noalloc_near_the_limit_allocates_nothing(lib):
    # 648 x 1266 uint8, 4 quadrants, cyclic: a workspace 35 KB short of the
    # 32 MiB scratch, so the last bytes of the array are used
    from paper_2411_07351_gb300 import _capi

    p = _plan(648, 1266, torch.uint8, "cyclic")
    assert (32 << 20) - 64 * 1024 < p.workspace_bytes <= (32 << 20)
    x = torch.from_numpy(inputs.uniform_u8(25, 648, 1266)).cuda()
    ref, got = _both(lib, p, x)  # also the warm-up of this shape
    assert torch.equal(ref, got)
    s = torch.cuda.current_stream().cuda_stream
    outs = [torch.full_like(ref, -1) for _ in range(3)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for o in outs:
        _capi.check(lib.fht_forward_noalloc(p._h, x.data_ptr(), x.stride(0), o.data_ptr(), s), "fht_forward_noalloc")
    torch.cuda.synchronize()
    # nothing was allocated by the calls: neither through torch nor by the driver
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0
    assert torch.cuda.mem_get_info()[0] == free0
    for o in outs:
        assert torch.equal(o, ref)
    # the device-side status word of the built-in scratch reads clean
    assert lib.fht_noalloc_status(torch.cuda.current_device(), s) == _capi.FHT_OK


def test_noalloc_rejects_plans_above_the_scratch_size(lib):
    from paper_2411_07351_gb300 import _capi

    p = _plan(4095, 4095, torch.float32, "extended")
    assert p.workspace_bytes > (32 << 20)
    x = torch.zeros((4095, 4095), dtype=torch.float32, device="cuda")
    out = p.new_output()
    st = lib.fht_forward_noalloc(p._h, x.data_ptr(), 4095, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == _capi.FHT_ERR_INVALID
    assert b"scratch" in lib.fht_last_error()
