"""GPU parity of the forward transform against the CPU oracle.

Integer inputs (uint8 -> int32, int32 -> int32) must be bit-exact.  Float32
must satisfy |H_gpu - H_fp64| <= 1e-5 * M element by element, where M is the
same transform of |I| in float64 (the L1 mass of the pattern); float64 must
satisfy the same bound at 1e-12.
"""
import numpy as np
import pytest
import torch

from paper_2411_07351_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_F64 = 1e-12


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_07351_gb300 import build as B

    B.build()
    import paper_2411_07351_gb300 as F

    return F


def _run(F, img_np, quads, boundary, split="T", **tun):
    x = torch.from_numpy(np.ascontiguousarray(img_np)).cuda()
    p = F.Plan(img_np.shape[0], img_np.shape[1], x.dtype, quads, boundary, split, **tun)
    p.check()
    out = p.forward(x)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _ob(orc, b):
    return orc.EXTENDED if b == "extended" else orc.CYCLIC


def _rule(orc, s):
    return orc.SPLIT_S if s == "S" else orc.SPLIT_T


def check_exact(F, orc, img, quads, boundary, split="T", **tun):
    got = _run(F, img, quads, boundary, split, **tun)
    ref = orc.fht(img.astype(np.int64), quads, _ob(orc, boundary), _rule(orc, split))
    assert got.shape == ref.shape
    bad = np.nonzero(got.astype(np.int64) != ref)[0]
    assert bad.size == 0, f"{bad.size} mismatches, first at {bad[:5]}: got {got[bad[:5]]} want {ref[bad[:5]]}"


def check_float(F, orc, img, quads, boundary, split="T", tol=TOL_F32, **tun):
    got = _run(F, img, quads, boundary, split, **tun).astype(np.float64)
    ref = orc.fht(img.astype(np.float64), quads, _ob(orc, boundary), _rule(orc, split))
    mass = orc.fht(np.abs(img.astype(np.float64)), quads, _ob(orc, boundary), _rule(orc, split))
    err = np.abs(got - ref)
    bound = tol * mass + 1e-30
    worst = int(np.argmax(err / bound))
    assert (err <= bound).all(), f"worst {err[worst]} vs bound {bound[worst]} at {worst}"


AWKWARD_H = [1, 2, 3, 5, 17, 63, 64, 65, 127, 129, 255, 257]
AWKWARD_W = [1, 2, 3, 4, 31, 33, 130]


@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_c1_257_exact(F, orc, boundary):
    img = inputs.c1_image()
    check_exact(F, orc, img, 1, boundary)
    check_exact(F, orc, img, 15, boundary)


def test_c1_matches_brute_force(F, orc):
    img = inputs.c1_image()
    got = _run(F, img, 1, "cyclic")
    ref = orc.brute(img.astype(np.int64), 1, orc.CYCLIC)
    assert np.array_equal(got.astype(np.int64), ref)


@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_awkward_sizes_u8(F, orc, boundary):
    for h in AWKWARD_H:
        for w in AWKWARD_W:
            img = inputs.uniform_u8(100 + h * 7 + w, h, w)
            check_exact(F, orc, img, 15, boundary)


@pytest.mark.parametrize("h,w", [(511, 300), (4095, 33), (4097, 17), (33, 4097), (1000, 1000), (1500, 2600)])
def test_larger_u8(F, orc, h, w):
    img = inputs.uniform_u8(h + w, h, w)
    check_exact(F, orc, img, 15, "cyclic")
    check_exact(F, orc, img, 15, "extended")


@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_split_s_u8(F, orc, boundary):
    for h, w in [(3, 5), (23, 45), (100, 64), (363, 90)]:
        img = inputs.uniform_u8(h * w, h, w)
        check_exact(F, orc, img, 15, boundary, "S")


@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_float32(F, orc, boundary):
    for h, w in [(1, 9), (13, 11), (64, 64), (65, 200), (300, 257), (700, 500)]:
        img = inputs.normal_f32(h + 3 * w, h, w)
        check_float(F, orc, img, 15, boundary)


def test_float64_and_int32(F, orc):
    rng = np.random.default_rng(0)
    for h, w in [(7, 3), (129, 77), (257, 100)]:
        img = rng.standard_normal((h, w))
        check_float(F, orc, img, 15, "extended", tol=TOL_F64)
        imi = rng.integers(-1000, 1000, (h, w)).astype(np.int32)
        check_exact(F, orc, imi, 15, "cyclic")


@pytest.mark.parametrize("fused_rows,tile_cols", [(1, 32), (2, 64), (8, 96), (32, 256), (64, 32)])
def test_tuning_knobs_same_result(F, orc, fused_rows, tile_cols):
    img = inputs.uniform_u8(7, 200, 150)
    check_exact(F, orc, img, 15, "extended", fused_rows=fused_rows, tile_cols=tile_cols)
    check_exact(F, orc, img, 15, "cyclic", fused_rows=fused_rows, tile_cols=tile_cols)


@pytest.mark.parametrize("tile_cols,threads", [(64, 512), (128, 512), (128, 256), (96, 512)])
def test_float_launch_shapes(F, orc, tile_cols, threads):
    # float inputs take the pipelined block pass at 512 threads and 64- or
    # 128-column tiles, the per-tile block pass otherwise: same result
    img = inputs.normal_f32(31, 700, 515)
    check_float(F, orc, img, 15, "extended", tile_cols=tile_cols, threads=threads)
    check_float(F, orc, img, 15, "cyclic", tile_cols=tile_cols, threads=threads)
    imi = inputs.uniform_u8(32, 300, 200).astype(np.int32) - 128
    check_exact(F, orc, imi, 15, "extended", tile_cols=tile_cols, threads=threads)


VTILE = dict(tile_cols=192, threads=256)


@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_register_tiled_blocks_u8(F, orc, boundary):
    """The register-tiled block launches (tiles of 192 columns, 256 threads):
    64-row roots (stored through the quadrant column map), blocks only (h a
    multiple of 64, one launch), blocks after a generic remainder launch,
    bands of every group size 2..64 blocks (a 4096-row band is the root),
    widths around the tile and narrow ones, every quadrant."""
    for h, w in [(64, 1), (64, 3), (64, 200), (128, 191), (128, 192), (128, 193), (65, 33), (200, 385),
                 (191, 64), (256, 17), (320, 450), (1000, 77), (1100, 30), (2100, 21), (4096, 13), (4095, 9),
                 (3071, 40)]:
        img = inputs.uniform_u8(1000 + h * 3 + w, h, w)
        check_exact(F, orc, img, 15, boundary, **VTILE)
        check_exact(F, orc, img, 1, boundary, **VTILE)


@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_register_tiled_blocks_f32_i32(F, orc, boundary):
    for h, w in [(64, 64), (129, 300), (700, 515), (4096, 65)]:
        img = inputs.normal_f32(77 + h + w, h, w)
        check_float(F, orc, img, 15, boundary, **VTILE)
    imi = inputs.uniform_u8(33, 300, 200).astype(np.int32) - 128
    check_exact(F, orc, imi, 15, boundary, **VTILE)


def test_register_tiled_pitched_input(F, orc):
    img = inputs.uniform_u8(19, 130, 71)
    big = torch.zeros((130, 100), dtype=torch.uint8)
    big[:, :71] = torch.from_numpy(img)
    x = big.cuda()[:, :71]
    p = F.Plan(130, 71, torch.uint8, 15, "extended", **VTILE)
    p.check()
    got = p.forward(x).cpu().numpy().astype(np.int64)
    assert np.array_equal(got, orc.fht(img.astype(np.int64), 15, orc.EXTENDED))


def test_pitched_input(F, orc):
    img = inputs.uniform_u8(9, 100, 70)
    big = torch.zeros((100, 96), dtype=torch.uint8)
    big[:, :70] = torch.from_numpy(img)
    x = big.cuda()[:, :70]
    assert x.stride(0) == 96
    p = F.Plan(100, 70, torch.uint8, 15, "extended")
    got = p.forward(x).cpu().numpy().astype(np.int64)
    assert np.array_equal(got, orc.fht(img.astype(np.int64), 15, orc.EXTENDED))


@pytest.mark.parametrize("boundary", ["extended", "cyclic"])
def test_c2_full_size_every_output(F, orc, boundary):
    """4095 x 4095 float32, four quadrants, in the plan the benchmark times:
    EVERY output against the oracle's recursion in FP64, with the L1 mass M
    (the same transform of |I|) as the scale of the tolerance."""
    img = inputs.c2_image()
    x = torch.from_numpy(img).cuda()
    p = F.Plan(4095, 4095, torch.float32, 15, boundary)
    out = p.forward(x)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    del out
    b = orc.EXTENDED if boundary == "extended" else orc.CYCLIC
    ref = orc.fht(img.astype(np.float64), 15, b)
    mass = orc.fht(np.abs(img.astype(np.float64)), 15, b)
    assert got.shape == ref.shape
    worst = 0.0
    for k in range(0, ref.size, 1 << 24):
        sl = slice(k, k + (1 << 24))
        err = np.abs(got[sl].astype(np.float64) - ref[sl])
        bad = err > TOL_F32 * mass[sl]
        assert not bad.any(), (k + int(np.argmax(bad)), float(err[bad].max()))
        worst = max(worst, float((err / np.maximum(mass[sl], 1e-300)).max()))
    assert worst <= TOL_F32


def test_repeat_deterministic(F):
    img = inputs.uniform_u8(3, 300, 300)
    a = _run(F, img, 15, "extended")
    b = _run(F, img, 15, "extended")
    assert np.array_equal(a, b)


def test_float_k_rounding(F, orc):
    """Plans with rounding='float' (Algorithm 1 read in floating point) match the
    oracle under the same rule, bit-exactly, at sizes where the rules differ."""
    orc.set_rounding(orc.ROUND_FLOAT)
    try:
        for h, w in [(23, 30), (45, 17), (181, 64), (725, 40)]:
            img = inputs.uniform_u8(h * 3 + w, h, w)
            x = torch.from_numpy(img).cuda()
            p = F.Plan(h, w, torch.uint8, 15, "extended", rounding="float")
            p.check()
            got = p.forward(x).cpu().numpy().astype(np.int64)
            assert np.array_equal(got, orc.fht(img.astype(np.int64), 15, orc.EXTENDED))
    finally:
        orc.set_rounding(orc.ROUND_EXACT)


@pytest.mark.parametrize("spine_chunk", [1, 2, 3, 100])
def test_spine_chunks_same_result(F, orc, spine_chunk):
    """The spine of a Split_T root summed in chunks (lower chunk tops first, as
    single parts of the chunk above) gives the same transform for every chunk size."""
    img = inputs.uniform_u8(2047 + spine_chunk, 2047, 300)
    check_exact(F, orc, img, 15, "cyclic", spine_chunk=spine_chunk)
    check_exact(F, orc, img, 15, "extended", spine_chunk=spine_chunk)
    imf = inputs.normal_f32(1500 + spine_chunk, 1500, 777)
    check_float(F, orc, imf, 15, "extended", spine_chunk=spine_chunk)


def test_largest_size_cyclic(F, orc):
    """h = 65535 (the largest supported): big parts of 32768, 16384 and 8192
    rows summed from 4096-row bands, then a chunked spine; whole output."""
    img = inputs.uniform_u8(65535, 65535, 2)
    check_exact(F, orc, img, 15, "cyclic")
    img2 = inputs.uniform_u8(2, 3, 65535)
    check_exact(F, orc, img2, 15, "cyclic")


@pytest.mark.parametrize("h,w", [(9000, 37), (12289, 5), (16500, 9)])
def test_taller_than_8192(F, orc, h, w):
    """Split_T roots whose power-of-two part is taller than the largest band
    (4096 rows): that part is summed from its bands first.  Cyclic: the whole
    output against the oracle; extended: sampled outputs against the definition."""
    img = inputs.uniform_u8(h * 31 + w, h, w)
    check_exact(F, orc, img, 15, "cyclic")
    x = torch.from_numpy(img).cuda()
    p = F.Plan(h, w, torch.uint8, 15, "extended")
    p.check()
    blocks = p.unpack(p.forward(x))
    rng = np.random.default_rng(h)
    k = 4000
    qs = rng.integers(0, 4, k)
    ts = np.array([rng.integers(0, blocks[q].shape[0]) for q in qs])
    xs = np.array([rng.integers(0, blocks[q].shape[1]) for q in qs])
    val, _ = orc.brute_at(img, qs, ts, xs, orc.EXTENDED)
    got = np.zeros(k, dtype=np.int64)
    for q in range(4):
        sel = np.nonzero(qs == q)[0]
        ti, xi = torch.from_numpy(ts[sel]).cuda(), torch.from_numpy(xs[sel]).cuda()
        got[sel] = blocks[q][ti, xi].cpu().numpy()
    assert np.array_equal(got, val.astype(np.int64))
    # every row of every quadrant sums to the image total
    total = int(img.astype(np.int64).sum())
    for b in blocks:
        assert (b.long().sum(1) == total).all()
    del blocks, x, p
    torch.cuda.empty_cache()


def test_workspace_status_cleared_by_forward(F, orc):
    """The workspace's device status word is cleared by every forward (the rest
    of the workspace may hold anything on entry) and stays FHT_OK when the
    staged spine's bounded waits all complete."""
    from paper_2411_07351_gb300 import _capi

    img = inputs.normal_f32(5, 1500, 700)
    x = torch.from_numpy(img).cuda()
    p = F.Plan(1500, 700, torch.float32, 15, "extended")
    out, ws = p.new_output(), p.new_workspace()
    ws.fill_(0xFF)  # garbage, including the status word
    p.forward(x, out, ws)
    lib = _capi.load()
    st = lib.fht_ws_status(ws.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == _capi.FHT_OK
    check_float(F, orc, img, 15, "extended")
