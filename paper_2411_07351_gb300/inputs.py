"""Seeded synthetic inputs for the five workloads (numpy PCG64).

These generators hold none of the transform's arithmetic; the tests, the
benchmark and the oracle all draw their inputs from here.  The paper uses no
dataset, so nothing is stood in for.

  c1  one 257 x 257 uint8 image, pixels i.i.d. U{0..255}               (seed 1)
  c2  one 4095 x 4095 float32 image, pixels i.i.d. N(0, 1)             (seed 2)
  c3  4096 binary uint8 edge maps, h, w ~ U{17..511} independently;
      Bernoulli(0.05) ones plus 20 width-1 Bresenham segments with
      uniform endpoints                                                (seed 3)
  c4  64 float32 images, h, w ~ U{200..600}, pixels U[0, 1), and target
      sinograms y ~ N(0, 1) of the packed 4-quadrant cyclic shape      (seeds 4, 5)
  c5  Poisson arrivals, 2000 req/s for 30 s; h, w = round(exp(U[ln 64,
      ln 4096])); uint8 with Bernoulli(0.1) non-zero pixels, values
      U{1..255}                                                        (seed 6)
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def c1_image(seed: int = 1) -> np.ndarray:
    return rng(seed).integers(0, 256, size=(257, 257), dtype=np.uint8)


def c2_image(seed: int = 2, h: int = 4095, w: int = 4095) -> np.ndarray:
    return rng(seed).standard_normal((h, w), dtype=np.float32)


def uniform_u8(seed: int, h: int, w: int) -> np.ndarray:
    return rng(seed).integers(0, 256, size=(h, w), dtype=np.uint8)


def normal_f32(seed: int, h: int, w: int) -> np.ndarray:
    return rng(seed).standard_normal((h, w), dtype=np.float32)


def _bresenham(img: np.ndarray, x0: int, y0: int, x1: int, y1: int) -> None:
    dx, dy = abs(x1 - x0), -abs(y1 - y0)
    sx, sy = (1 if x0 < x1 else -1), (1 if y0 < y1 else -1)
    err = dx + dy
    while True:
        img[y0, x0] = 1
        if x0 == x1 and y0 == y1:
            break
        e2 = 2 * err
        if e2 >= dy:
            err += dy
            x0 += sx
        if e2 <= dx:
            err += dx
            y0 += sy


def edge_map(g: np.random.Generator, h: int, w: int, density: float = 0.05, segments: int = 20) -> np.ndarray:
    img = (g.random((h, w)) < density).astype(np.uint8)
    for _ in range(segments):
        x0, x1 = g.integers(0, w, 2)
        y0, y1 = g.integers(0, h, 2)
        _bresenham(img, int(x0), int(y0), int(x1), int(y1))
    return img


def c3_batch(seed: int = 3, count: int = 4096, lo: int = 17, hi: int = 511) -> list[np.ndarray]:
    g = rng(seed)
    sizes = g.integers(lo, hi + 1, size=(count, 2))
    return [edge_map(g, int(h), int(w)) for h, w in sizes]


def c4_batch(seed: int = 4, count: int = 64, lo: int = 200, hi: int = 600) -> list[np.ndarray]:
    g = rng(seed)
    sizes = g.integers(lo, hi + 1, size=(count, 2))
    return [g.random((int(h), int(w)), dtype=np.float32) for h, w in sizes]


def c4_targets(images: list[np.ndarray], seed: int = 5) -> list[np.ndarray]:
    """Targets y of the packed four-quadrant cyclic output shape of each image."""
    g = rng(seed)
    out = []
    for im in images:
        h, w = im.shape
        out.append(g.standard_normal(2 * h * w + 2 * w * h, dtype=np.float32))
    return out


def c5_requests(seed: int = 6, rate: float = 2000.0, duration: float = 30.0, lo: int = 64, hi: int = 4096,
                max_requests: int | None = None):
    """Yields (arrival_time_s, h, w, image) lazily; images drawn at yield time."""
    g = rng(seed)
    t = 0.0
    k = 0
    while True:
        t += g.exponential(1.0 / rate)
        if t > duration or (max_requests is not None and k >= max_requests):
            return
        h = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        w = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        nz = g.random((h, w)) < 0.1
        img = np.where(nz, g.integers(1, 256, size=(h, w)), 0).astype(np.uint8)
        k += 1
        yield t, h, w, img
