"""Pin of the oracle's sampled checker ``brute_at`` (the definition of the
Hough value, Section 3 with Algorithm 2's patterns, evaluated at chosen
outputs).

``brute_at`` is what the full-size GPU tests compare against when the whole
transform is too large for the recursion, so it is pinned here against the
two pinned forms of the oracle at EVERY output of small images: the recursion
of Algorithm 1 (``fht``) and the explicit pattern sums (``brute``).  Its value
and its L1 mass (the same sum over |I|) are both checked, for all four
quadrants, both boundaries, both split rules, and sizes that include the
degenerate ones (h = 1, w = 1) and the extended padding columns.
"""
import numpy as np
import pytest

QALL = 15


def _all_outputs(orc, h, w, boundary):
    qs, ts, xs = [], [], []
    for q, (n, width) in zip([q for q in range(4)], orc.out_shape(h, w, QALL, boundary)):
        t, x = np.meshgrid(np.arange(n), np.arange(width), indexing="ij")
        qs.append(np.full(t.size, q))
        ts.append(t.ravel())
        xs.append(x.ravel())
    return np.concatenate(qs), np.concatenate(ts), np.concatenate(xs)


def _sizes():
    rng = np.random.default_rng(11)
    fixed = [(1, 1), (1, 7), (7, 1), (2, 3), (3, 2), (13, 11), (17, 5), (40, 40), (33, 9), (9, 33)]
    drawn = [tuple(int(v) for v in rng.integers(1, 41, size=2)) for _ in range(10)]
    return fixed + drawn


@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("rule", [0, 1])
def test_brute_at_equals_recursion_everywhere(orc, boundary, rule):
    rng = np.random.default_rng(100 + 2 * boundary + rule)
    for h, w in _sizes():
        img = rng.integers(-50, 51, size=(h, w)).astype(np.float64)
        qs, ts, xs = _all_outputs(orc, h, w, boundary)
        val, mass = orc.brute_at(img, qs, ts, xs, boundary, rule)
        # integer-valued doubles: every sum below 2^53 is exact, so equality is exact
        ref = orc.fht(img.astype(np.int64), QALL, boundary, rule).astype(np.float64)
        ref_mass = orc.fht(np.abs(img).astype(np.int64), QALL, boundary, rule).astype(np.float64)
        np.testing.assert_array_equal(val, ref, err_msg=f"value {h}x{w}")
        np.testing.assert_array_equal(mass, ref_mass, err_msg=f"mass {h}x{w}")


@pytest.mark.parametrize("boundary", [0, 1])
def test_brute_at_equals_pattern_sums(orc, boundary):
    # against O2 (explicit patterns) on float data, where the sums are not exact:
    # the same additions in the same order (y ascending) give the same rounding
    rng = np.random.default_rng(7 + boundary)
    for h, w in [(5, 8), (12, 12), (23, 19)]:
        img = rng.standard_normal((h, w))
        qs, ts, xs = _all_outputs(orc, h, w, boundary)
        val, _ = orc.brute_at(img, qs, ts, xs, boundary)
        ref = orc.brute(img, QALL, boundary)
        np.testing.assert_allclose(val, ref, rtol=0, atol=1e-12)


def test_brute_at_transposed_index(orc):
    # Q2 of an image is Q0 of its transpose (R5): a mistake in the transposed
    # index of the sampled checker shows here on a non-square image
    rng = np.random.default_rng(5)
    img = rng.integers(0, 9, size=(6, 11)).astype(np.float64)
    qs, ts, xs = _all_outputs(orc, 11, 6, 0)
    q0 = qs < 2
    v_t, _ = orc.brute_at(img.T.copy(), qs[q0], ts[q0], xs[q0], 0)
    qs2, ts2, xs2 = _all_outputs(orc, 6, 11, 0)
    q2 = qs2 >= 2
    v, _ = orc.brute_at(img, qs2[q2], ts2[q2], xs2[q2], 0)
    np.testing.assert_array_equal(v, v_t)


def test_parallel_digests_match_direct_runs(orc):
    # the spawned-process driver used by the whole-workload GPU checks returns,
    # per image, the digest of exactly what the oracle computes in-process
    from oracle import parallel

    rng = np.random.default_rng(3)
    imgs = [rng.integers(0, 256, size=(int(h), int(w)), dtype=np.uint8)
            for h, w in rng.integers(1, 60, size=(9, 2))]
    got = parallel.int32_digests(imgs, QALL, 0, procs=3)
    assert sorted(got) == list(range(len(imgs)))
    for k, im in enumerate(imgs):
        assert got[k] == parallel.digest(orc.fht(im.astype(np.int64), QALL, 0).astype(np.int32))
    # a changed element changes the digest
    ref = orc.fht(imgs[0].astype(np.int64), QALL, 0).astype(np.int32)
    ref[len(ref) // 2] += 1
    assert parallel.digest(ref) != got[0]
