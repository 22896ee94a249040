"""Plain CPU oracle for the generalised Brady-Yong fast Hough transform.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2411_07351_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``fht_oracle.c`` (single-threaded C, int64 / double),
compiled here with gcc into ``liboracle.so`` and called through ctypes.  Each
C function cites the passage of the paper it follows:

* ``pattern``        -- Algorithm 2 (FHT2D_Pattern), Section 3.
* ``fht``            -- Algorithm 1 (FHT2D), Section 3, in the row-split
                        orientation (the paper's algorithm on the transposed
                        image); quadrants and the EXTENDED boundary as
                        documented in the C file.
* ``brute``          -- the definition: sums along every pattern of Algorithm 2.
* ``brady_yong``     -- the classical power-of-two transform (Sections 2-3).
* ``adjoint``        -- the transpose of Algorithm 1's merge (back-projection).
* ``pattern_error``  -- the orthotropic error E(n) of Section 4.
* ``adds``           -- the addition count f(n) of Theorem 1's proof.

Every function here is pinned by ``tests/test_oracle*.py`` against values the
paper prints, closed forms from the paper and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fht_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SPLIT_T, SPLIT_S = 0, 1
CYCLIC, EXTENDED = 0, 1


def build(force: bool = False) -> str:
    """Compile ``fht_oracle.c`` into ``liboracle.so`` (gcc, -O2, no -march)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i32, i64, u32, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p
            lib.orc_split.argtypes = [i32, i32, vp]
            lib.orc_round_half_even.argtypes = [i64, i64]
            lib.orc_round_half_even.restype = i64
            lib.orc_pattern.argtypes = [i32, i32, i32, vp]
            lib.orc_pattern_error_num.argtypes = [i32, i32]
            lib.orc_pattern_error_num.restype = i64
            lib.orc_tree_nonleaf_sum.argtypes = [i32, i32]
            lib.orc_tree_nonleaf_sum.restype = i64
            lib.orc_out_elems.argtypes = [i32, i32, u32, i32]
            lib.orc_out_elems.restype = i64
            for name in ("orc_fht_i64", "orc_fht_f64", "orc_brute_i64", "orc_brute_f64",
                         "orc_adjoint_f64", "orc_adjoint_brute_f64"):
                getattr(lib, name).argtypes = [i32, i32, vp, u32, i32, i32, vp]
            lib.orc_brute_at_f64.argtypes = [i32, i32, vp, i32, i32, i64, vp, vp, vp, vp, vp]
            lib.orc_set_rounding.argtypes = [i32]
            lib.orc_child_slope.argtypes = [i32, i32, i32]
            lib.orc_child_slope.restype = i32
            lib.orc_brady_yong_i64.argtypes = [i32, i32, vp, vp]
            lib.orc_brady_yong_i64.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


ROUND_EXACT, ROUND_FLOAT = 0, 1


def set_rounding(rule: int):
    """Child-slope rounding for every later call: ROUND_EXACT (ties to even on the
    exact rational, the default) or ROUND_FLOAT (k = (n_P - 1)/(n - 1) in double,
    then rint(t k))."""
    _load().orc_set_rounding(rule)


def child_slope(n: int, ni: int, t: int) -> int:
    """[t (ni - 1)/(n - 1)] under the current rounding rule."""
    return int(_load().orc_child_slope(n, ni, t))


def split(n: int, rule: int = SPLIT_T) -> tuple[int, int]:
    out = np.zeros(2, np.int32)
    _load().orc_split(n, rule, _ptr(out))
    return int(out[0]), int(out[1])


def round_half_even(a: int, d: int) -> int:
    return int(_load().orc_round_half_even(a, d))


def pattern(n: int, t: int, rule: int = SPLIT_T) -> np.ndarray:
    """Algorithm 2: pat(n, t) as an int32 vector of length n."""
    if not (n >= 1 and 0 <= t < n):
        raise ValueError("need n >= 1 and 0 <= t < n")
    out = np.zeros(n, np.int32)
    _load().orc_pattern(n, t, rule, _ptr(out))
    return out


def pattern_error_num(n: int, rule: int = SPLIT_T) -> int:
    """Exact numerator of E(n): E(n) = pattern_error_num(n) / (n - 1)."""
    return int(_load().orc_pattern_error_num(n, rule))


def pattern_error(n: int, rule: int = SPLIT_T) -> float:
    return 0.0 if n <= 1 else pattern_error_num(n, rule) / (n - 1)


def tree_nonleaf_sum(n: int, rule: int = SPLIT_T) -> int:
    return int(_load().orc_tree_nonleaf_sum(n, rule))


def adds(n: int, rule: int = SPLIT_T) -> int:
    """Theorem 1: additions of the n x n transform, f(n) = n * sum of non-leaf node values."""
    return n * tree_nonleaf_sum(n, rule)


def out_shape(h: int, w: int, quads: int, boundary: int) -> list[tuple[int, int]]:
    shapes = []
    for q in range(4):
        if quads & (1 << q):
            n, length = (h, w) if q < 2 else (w, h)
            shapes.append((n, length + n - 1 if boundary == EXTENDED else length))
    return shapes


def out_elems(h: int, w: int, quads: int, boundary: int) -> int:
    return int(_load().orc_out_elems(h, w, quads, boundary))


def _run(fn_i64, fn_f64, img, quads, boundary, rule, exact):
    img = np.asarray(img)
    h, w = img.shape
    n_out = out_elems(h, w, quads, boundary)
    if exact:
        src = np.ascontiguousarray(img, dtype=np.int64)
        out = np.zeros(n_out, np.int64)
        fn_i64(h, w, _ptr(src), quads, boundary, rule, _ptr(out))
    else:
        src = np.ascontiguousarray(img, dtype=np.float64)
        out = np.zeros(n_out, np.float64)
        fn_f64(h, w, _ptr(src), quads, boundary, rule, _ptr(out))
    return out


def _is_exact(img) -> bool:
    return np.issubdtype(np.asarray(img).dtype, np.integer)


def fht(img, quads: int = 1, boundary: int = CYCLIC, rule: int = SPLIT_T) -> np.ndarray:
    """O1, Algorithm 1.  Integer images in int64, float images in float64.

    Returns the packed flat output (quadrants Q0..Q3 that are set in ``quads``).
    """
    lib = _load()
    return _run(lib.orc_fht_i64, lib.orc_fht_f64, img, quads, boundary, rule, _is_exact(img))


def brute(img, quads: int = 1, boundary: int = CYCLIC, rule: int = SPLIT_T) -> np.ndarray:
    """O2: explicit pattern sums (tiny sizes only: O(n^2 W) per quadrant)."""
    lib = _load()
    return _run(lib.orc_brute_i64, lib.orc_brute_f64, img, quads, boundary, rule, _is_exact(img))


def unpack(flat: np.ndarray, h: int, w: int, quads: int, boundary: int) -> list[np.ndarray]:
    res, off = [], 0
    for n, width in out_shape(h, w, quads, boundary):
        res.append(flat[off:off + n * width].reshape(n, width))
        off += n * width
    return res


def adjoint(gout, h: int, w: int, quads: int = 1, boundary: int = CYCLIC, rule: int = SPLIT_T,
            brute_force: bool = False) -> np.ndarray:
    """Transpose of the packed transform, float64: returns the h x w image gradient."""
    lib = _load()
    g = np.ascontiguousarray(np.asarray(gout, dtype=np.float64).reshape(-1))
    if g.size != out_elems(h, w, quads, boundary):
        raise ValueError("gout has the wrong number of elements")
    out = np.zeros((h, w), np.float64)
    fn = lib.orc_adjoint_brute_f64 if brute_force else lib.orc_adjoint_f64
    fn(h, w, _ptr(g), quads, boundary, rule, _ptr(out))
    return out


def brute_at(img, qs, ts, xs, boundary: int = CYCLIC, rule: int = SPLIT_T):
    """Definition evaluated at sampled outputs (q, t, x): returns (values, L1 masses), float64."""
    src = np.ascontiguousarray(np.asarray(img), dtype=np.float64)
    h, w = src.shape
    qs = np.ascontiguousarray(qs, dtype=np.int32)
    ts = np.ascontiguousarray(ts, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    val = np.zeros(len(qs), np.float64)
    mass = np.zeros(len(qs), np.float64)
    _load().orc_brute_at_f64(h, w, _ptr(src), boundary, rule, len(qs), _ptr(qs), _ptr(ts), _ptr(xs),
                             _ptr(val), _ptr(mass))
    return val, mass


def brady_yong(img) -> np.ndarray:
    """Classical Brady-Yong (Q0, cyclic) for a 2^q-row integer image."""
    src = np.ascontiguousarray(np.asarray(img), dtype=np.int64)
    n, width = src.shape
    out = np.zeros_like(src)
    if _load().orc_brady_yong_i64(n, width, _ptr(src), _ptr(out)) != 0:
        raise ValueError("Brady-Yong needs a power-of-two number of rows")
    return out
