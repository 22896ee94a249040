"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them compares the oracle with
itself through a retyped formula: they use hand-derived tables (Section 3,
Algorithms 1-2), the brute-force definition (sums along Algorithm 2's
patterns), the classical Brady-Yong transform (Sections 2-3), closed forms
(Theorem 1), the Theorem 2 bound, and invariants of any line-sum transform.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _worked():
    tables, pats = [], []
    with open(os.path.join(GOLDEN, "worked_tables.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "pattern":
                pats.append((int(parts[1]), int(parts[2]), [int(v) for v in parts[3:]]))
            else:
                tables.append(tuple(int(v) for v in parts))
    return tables, pats


def test_split_rules(orc):
    # Section 3: Split_S bisects, Split_T cuts off the largest power of two below n.
    assert [orc.split(n) for n in (2, 3, 4, 5, 7, 12, 17, 4095)] == [
        (1, 1), (2, 1), (2, 2), (4, 1), (4, 3), (8, 4), (16, 1), (2048, 2047)]
    assert [orc.split(n, orc.SPLIT_S) for n in (2, 3, 7, 4095)] == [(1, 1), (1, 2), (3, 4), (2047, 2048)]


def test_round_half_even(orc):
    assert [orc.round_half_even(a, 2) for a in range(8)] == [0, 0, 1, 2, 2, 2, 3, 4]
    assert orc.round_half_even(35, 12) == 3 and orc.round_half_even(20, 12) == 2
    assert orc.round_half_even(15 * 8, 16) == 8  # 7.5 -> 8


def test_worked_tables_and_pattern(orc):
    tables, pats = _worked()
    for n, t, t1, t2, s in tables:
        n0, n1 = orc.split(n)
        assert orc.round_half_even(t * (n0 - 1), n - 1) == t1
        assert orc.round_half_even(t * (n1 - 1), n - 1) == t2
        assert t - t2 == s
        # Algorithm 2: the right part of pat(n,t) starts at pat(n1,t2)[0] + s = s
        assert orc.pattern(n, t)[n0] == s
    for n, t, ref in pats:
        assert list(orc.pattern(n, t)) == ref


@pytest.mark.parametrize("rule", [0, 1])
def test_pattern_shape(orc, rule):
    # Dyadic patterns are digital lines: start at 0, end at t, steps in {0, 1}.
    for n in range(1, 130):
        for t in range(n):
            p = orc.pattern(n, t, rule)
            assert p[0] == 0 and p[-1] == t
            d = np.diff(p)
            assert ((d == 0) | (d == 1)).all()


def test_small_n_errors(orc):
    # Hand-checkable small cases of E_T(n) (half-to-even rounding).
    expect = {3: .5, 5: .5, 6: .6, 7: 2 / 3, 9: .75, 11: .7, 13: .75, 17: .875, 19: 1.0}
    for n, e in expect.items():
        assert orc.pattern_error(n) == pytest.approx(e, abs=1e-12)


def test_karpenko_power_of_two_error(orc):
    # Section 2 quotes log2(n)/6 for even q and log2(n)/6 - 1/18 for odd q as the
    # maximal error of the 2^q patterns.  Under the line y = x t/(n-1) the even
    # case is exact and the odd case is an upper bound that is approached.
    for q in range(2, 11):
        e = orc.pattern_error(2 ** q)
        if q % 2 == 0:
            assert e == pytest.approx(q / 6, abs=1e-12)
        else:
            assert e <= q / 6 - 1 / 18 + 1e-12
            assert e > q / 6 - 1 / 18 - 0.07


def _rand_img(rng, h, w, exact):
    if exact:
        return rng.integers(0, 256, (h, w)).astype(np.int64)
    return rng.standard_normal((h, w))


@pytest.mark.parametrize("rule", [0, 1])
def test_recursion_equals_brute_force_all_small(orc, rule):
    # Pin 1: Algorithm 1 (O1) == sums along Algorithm 2's patterns (O2), exactly,
    # for every h, w in [1, 16] (and both boundaries, all quadrants).
    rng = np.random.default_rng(11 + rule)
    for h in range(1, 17):
        for w in range(1, 17):
            img = _rand_img(rng, h, w, True)
            for b in (orc.CYCLIC, orc.EXTENDED):
                a = orc.fht(img, 15, b, rule)
                c = orc.brute(img, 15, b, rule)
                assert np.array_equal(a, c), (h, w, b)


def test_recursion_equals_brute_force_random(orc):
    rng = np.random.default_rng(5)
    for _ in range(12):
        h, w = rng.integers(1, 65, 2)
        img = _rand_img(rng, int(h), int(w), False)
        for b in (orc.CYCLIC, orc.EXTENDED):
            a = orc.fht(img, 15, b)
            c = orc.brute(img, 15, b)
            assert np.allclose(a, c, rtol=0, atol=1e-9)
    img = _rand_img(rng, 13, 11, True)
    assert np.array_equal(orc.fht(img, 15, 1), orc.brute(img, 15, 1))


def test_brady_yong_power_of_two(orc):
    # Pin 2: both variants coincide with Brady-Yong for n = 2^q (Section 3).
    rng = np.random.default_rng(2)
    for q in range(0, 9):
        n = 2 ** q
        for width in (1, 3, 37, 64):
            img = rng.integers(0, 256, (n, width)).astype(np.int64)
            by = orc.brady_yong(img)
            for rule in (0, 1):
                assert np.array_equal(orc.fht(img, 1, orc.CYCLIC, rule).reshape(n, width), by)


def test_slope_zero_and_last_slope(orc):
    # Pin 3: pat(h, 0) = 0, so row 0 holds the column sums.
    # Pin 4: pat(h, h-1)[y] = y, so the last row sums the 45-degree diagonal.
    rng = np.random.default_rng(3)
    for h, w in [(1, 5), (2, 2), (5, 9), (17, 17), (33, 20), (100, 7)]:
        img = rng.integers(0, 256, (h, w)).astype(np.int64)
        for b in (orc.CYCLIC, orc.EXTENDED):
            (H,) = orc.unpack(orc.fht(img, 1, b), h, w, 1, b)
            W = H.shape[1]
            pad = np.zeros((h, W), np.int64)
            pad[:, :w] = img
            assert np.array_equal(H[0], pad.sum(0))
            diag = np.array([sum(pad[y, (x + y) % W] for y in range(h)) for x in range(W)])
            assert np.array_equal(H[h - 1], diag)
            (H1,) = orc.unpack(orc.fht(img, 2, b), h, w, 2, b)
            adiag = np.array([sum(pad[y, (x - y) % W] for y in range(h)) for x in range(W)])
            assert np.array_equal(H1[h - 1], adiag)


def test_mass_and_linearity(orc):
    # Pin 5: every slope row of every quadrant sums to the image mass.
    # Pin 6: linearity, exact in integers.
    rng = np.random.default_rng(4)
    for h, w in [(7, 5), (23, 31), (64, 3), (45, 45)]:
        a = rng.integers(0, 256, (h, w)).astype(np.int64)
        c = rng.integers(0, 256, (h, w)).astype(np.int64)
        for b in (orc.CYCLIC, orc.EXTENDED):
            for Hq in orc.unpack(orc.fht(a, 15, b), h, w, 15, b):
                assert (Hq.sum(1) == a.sum()).all()
            lhs = orc.fht(3 * a - 2 * c, 15, b)
            assert np.array_equal(lhs, 3 * orc.fht(a, 15, b) - 2 * orc.fht(c, 15, b))


def test_extended_is_non_wrapping_line_sum(orc):
    # EXTENDED boundary: output column x in [0, w) is the sum along the pattern
    # started at x with no wrap; columns x in [w, W) are the lines that enter
    # from the left, started at x - W.  Written with explicit bounds, no modulo.
    rng = np.random.default_rng(6)
    for h, w in [(5, 4), (9, 13), (17, 6)]:
        img = rng.integers(0, 256, (h, w)).astype(np.int64)
        W = w + h - 1
        H0, H1, H2, H3 = orc.unpack(orc.fht(img, 15, orc.EXTENDED), h, w, 15, orc.EXTENDED)
        for t in range(h):
            p = orc.pattern(h, t)
            for x in range(W):
                start = x if x < w else x - W
                s0 = sum(img[y, start + p[y]] for y in range(h) if 0 <= start + p[y] < w)
                assert H0[t, x] == s0
                # Q1 runs leftwards from column x; a wrap would only reach padding.
                s1 = sum(img[y, x - p[y]] for y in range(h) if 0 <= x - p[y] < w)
                assert H1[t, x] == s1
        imgT = img.T.copy()
        (G0, G1) = orc.unpack(orc.fht(imgT, 3, orc.EXTENDED), w, h, 3, orc.EXTENDED)
        assert np.array_equal(H2, G0) and np.array_equal(H3, G1)


def test_quadrant_symmetries(orc):
    # Q1 is the mirror of Q0 of the mirrored image (cyclic, x -> W-1-x);
    # Q2/Q3 are Q0/Q1 of the transposed image.
    rng = np.random.default_rng(7)
    for h, w in [(6, 9), (13, 11), (32, 5)]:
        img = rng.integers(0, 256, (h, w)).astype(np.int64)
        H0, H1, H2, H3 = orc.unpack(orc.fht(img, 15, orc.CYCLIC), h, w, 15, orc.CYCLIC)
        (M0,) = orc.unpack(orc.fht(img[:, ::-1], 1, orc.CYCLIC), h, w, 1, orc.CYCLIC)
        assert np.array_equal(H1, M0[:, ::-1])
        (T0, T1) = orc.unpack(orc.fht(img.T, 3, orc.CYCLIC), w, h, 3, orc.CYCLIC)
        assert np.array_equal(H2, T0) and np.array_equal(H3, T1)


def test_degenerate_sizes(orc):
    # h = 1: the transform is the identity (Algorithm 1's base case).
    # w = 1: every shift is mod 1, so every slope gives the column sum.
    rng = np.random.default_rng(8)
    img = rng.integers(0, 256, (1, 9)).astype(np.int64)
    assert np.array_equal(orc.fht(img, 1), img.reshape(-1))
    img = rng.integers(0, 256, (13, 1)).astype(np.int64)
    assert (orc.fht(img, 1) == img.sum()).all()


def test_theorem1_counts(orc):
    # Theorem 1: f_S closed form; f_T at 2^k + 1; sharp constants at n = 3, 17.
    for n in range(2, 4097):
        fl = int(math.floor(math.log2(n)))
        assert orc.adds(n, orc.SPLIT_S) == (fl + 2) * n * n - 2 ** (fl + 1) * n
    for k in range(1, 12):
        n = 2 ** k + 1
        assert orc.adds(n) == n * (n + k * 2 ** k)
    rs = [orc.adds(n, orc.SPLIT_S) / (n * n * math.log2(n)) for n in range(2, 4097)]
    rt = [orc.adds(n) / (n * n * math.log2(n)) for n in range(2, 4097)]
    assert int(np.argmax(rs)) + 2 == 3 and max(rs) == pytest.approx(5 * math.log(2, 3) / 3, rel=1e-12)
    assert int(np.argmax(rt)) + 2 == 17 and max(rt) == pytest.approx(81 * math.log(2, 17) / 17, rel=1e-12)
    assert max(rs) < 1.052 and max(rt) < 1.166


def test_adjoint(orc):
    # Pin 10: <Hx, y> = <x, H^T y>; recursion adjoint == brute-force back-projection;
    # H^T of a one-hot Hough image is the indicator of one pattern.
    rng = np.random.default_rng(9)
    for h, w in [(13, 11), (8, 8), (17, 5), (1, 4), (6, 1)]:
        for b in (orc.CYCLIC, orc.EXTENDED):
            x = rng.standard_normal((h, w))
            y = rng.standard_normal(orc.out_elems(h, w, 15, b))
            hx = orc.fht(x, 15, b)
            hty = orc.adjoint(y, h, w, 15, b)
            assert np.dot(hx, y) == pytest.approx(np.sum(x * hty), rel=1e-12, abs=1e-9)
            assert np.allclose(hty, orc.adjoint(y, h, w, 15, b, brute_force=True), atol=1e-9)
    h, w, t, x0 = 13, 11, 5, 3
    g = np.zeros(h * w)
    g[t * w + x0] = 1.0
    img = orc.adjoint(g, h, w, 1, orc.CYCLIC)
    p = orc.pattern(h, t)
    ref = np.zeros((h, w))
    for yy in range(h):
        ref[yy, (x0 + p[yy]) % w] = 1
    assert np.array_equal(img, ref)
