"""GPU adjoint (back-projection) against the CPU oracle, the dot-product test,
FP64 finite differences through autograd, and the 64-image training-step
workload (float32 images of 200..600 pixels a side)."""
import numpy as np
import pytest
import torch

from paper_2411_07351_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_07351_gb300 import build as B

    B.build()
    import paper_2411_07351_gb300 as F

    return F


def _ob(orc, b):
    return orc.EXTENDED if b == "extended" else orc.CYCLIC


@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_adjoint_matches_oracle(F, orc, boundary, dtype, tol):
    rng = np.random.default_rng(3)
    for h, w in [(1, 1), (1, 7), (9, 1), (13, 11), (64, 65), (65, 64), (129, 200), (257, 100)]:
        p = F.Plan(h, w, dtype, 15, boundary)
        p.check()
        g = rng.standard_normal(p.out_elems)
        got = p.adjoint(torch.from_numpy(g).to(dtype).cuda()).cpu().double().numpy()
        g_in = g.astype(np.float32).astype(np.float64) if dtype == torch.float32 else g
        ref = orc.adjoint(g_in, h, w, 15, _ob(orc, boundary))
        mass = orc.adjoint(np.abs(g_in), h, w, 15, _ob(orc, boundary))
        err = np.abs(got - ref)
        assert (err <= tol * mass + 1e-300).all(), (h, w, float((err / (mass + 1e-300)).max()))


@pytest.mark.parametrize("boundary", ["cyclic", "extended"])
def test_adjoint_large_default_plan(F, orc, boundary):
    """A float32 plan large enough for the register-tiled forward launch shape
    (tile 192, 256 threads): the adjoint, which shares the plan's tile width
    and CTA size, against the oracle element by element."""
    h, w = 2100, 2050
    p = F.Plan(h, w, torch.float32, 15, boundary, with_adjoint=True)
    assert p.info.tile_cols == 192
    p.check()
    g = np.random.default_rng(5).standard_normal(p.out_elems).astype(np.float32).astype(np.float64)
    got = p.adjoint(torch.from_numpy(g).float().cuda()).cpu().double().numpy()
    ref = orc.adjoint(g, h, w, 15, _ob(orc, boundary))
    mass = orc.adjoint(np.abs(g), h, w, 15, _ob(orc, boundary))
    err = np.abs(got - ref)
    assert (err <= 1e-5 * mass + 1e-300).all(), float((err / (mass + 1e-300)).max())


def test_adjoint_integer_exact(F, orc):
    rng = np.random.default_rng(4)
    for h, w, b in [(31, 17, "cyclic"), (70, 66, "extended")]:
        p = F.Plan(h, w, torch.uint8, 15, b)
        g = rng.integers(-50, 50, p.out_elems).astype(np.int32)
        got = p.adjoint(torch.from_numpy(g).cuda()).cpu().numpy().astype(np.int64)
        ref = orc.adjoint(g.astype(np.float64), h, w, 15, _ob(orc, b))
        assert np.array_equal(got, ref.astype(np.int64))


@pytest.mark.parametrize("split", ["T", "S"])
def test_dot_product(F, split):
    # <Hx, y> = <x, H^T y> in FP64, for every quadrant set and boundary
    g = torch.Generator(device="cuda").manual_seed(0)
    for h, w in [(13, 11), (100, 37), (300, 301)]:
        for b in ("cyclic", "extended"):
            for quads in (1, 2, 4, 8, 15):
                p = F.Plan(h, w, torch.float64, quads, b, split)
                x = torch.randn((h, w), dtype=torch.float64, device="cuda", generator=g)
                y = torch.randn(p.out_elems, dtype=torch.float64, device="cuda", generator=g)
                lhs = torch.dot(p.forward(x), y).item()
                rhs = torch.sum(x * p.adjoint(y)).item()
                scale = torch.dot(p.forward(x.abs()), y.abs()).item()
                assert abs(lhs - rhs) <= 1e-12 * scale


def test_gradcheck_fp64_13x11(F):
    from paper_2411_07351_gb300.autograd import fht

    x = torch.randn((13, 11), dtype=torch.float64, device="cuda", requires_grad=True)
    for b in ("cyclic", "extended"):
        assert torch.autograd.gradcheck(lambda t: fht(t, 15, b), (x,), eps=1e-6, atol=1e-5, rtol=1e-5)


def test_finite_difference_loss_13x11(F, orc):
    # FP64 central differences of 0.5 ||H x - y||^2 agree with the adjoint to 1e-5
    from paper_2411_07351_gb300.autograd import fht

    rng = np.random.default_rng(5)
    x0 = rng.standard_normal((13, 11))
    y = rng.standard_normal(orc.out_elems(13, 11, 15, orc.CYCLIC))
    xt = torch.from_numpy(x0).cuda().requires_grad_(True)
    yt = torch.from_numpy(y).cuda()
    loss = 0.5 * ((fht(xt, 15, "cyclic") - yt) ** 2).sum()
    loss.backward()
    grad = xt.grad.cpu().numpy()

    def f(xx):
        return 0.5 * np.sum((orc.fht(xx, 15, orc.CYCLIC) - y) ** 2)

    eps = 1e-6
    for idx in [(0, 0), (6, 5), (12, 10), (3, 9)]:
        e = np.zeros_like(x0)
        e[idx] = eps
        fd = (f(x0 + e) - f(x0 - e)) / (2 * eps)
        assert abs(fd - grad[idx]) <= 1e-5 * max(1.0, abs(fd))


def test_c4_training_step(F, orc):
    """64 float32 images (h, w in [200, 600]), loss 0.5 ||FHT(x) - y||^2 over the
    packed 4-quadrant cyclic output; gradients = H^T (H x - y), checked against
    the FP64 oracle on a sample of images."""
    from paper_2411_07351_gb300.autograd import fht

    imgs = inputs.c4_batch()
    ys = inputs.c4_targets(imgs)
    xs = [torch.from_numpy(im).cuda().requires_grad_(True) for im in imgs]
    loss = 0
    for x, y in zip(xs, ys):
        loss = loss + 0.5 * ((fht(x, 15, "cyclic") - torch.from_numpy(y).cuda()) ** 2).sum()
    loss.backward()
    for k in (0, 17, 63):
        im, y = imgs[k].astype(np.float64), ys[k].astype(np.float64)
        h, w = im.shape
        r = orc.fht(im, 15, orc.CYCLIC) - y
        ref = orc.adjoint(r, h, w, 15, orc.CYCLIC)
        mass = orc.adjoint(orc.fht(np.abs(im), 15, orc.CYCLIC) + np.abs(y), h, w, 15, orc.CYCLIC)
        got = xs[k].grad.cpu().double().numpy()
        assert (np.abs(got - ref) <= 1e-5 * mass).all()
