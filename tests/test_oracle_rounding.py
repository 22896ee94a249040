"""The floating-point reading of Algorithm 1's child slopes (k_P computed as a
double, then t k_P rounded): it may differ from the exact rule only where
t (n_P - 1)/(n - 1) is exactly a half-integer, and the oracle's recursion and
brute force agree under it."""
import numpy as np
import pytest


@pytest.fixture
def orc_float(orc):
    orc.set_rounding(orc.ROUND_FLOAT)
    yield orc
    orc.set_rounding(orc.ROUND_EXACT)


def test_float_rule_differs_only_at_ties(orc_float):
    orc = orc_float
    diffs, first = 0, None
    for n in range(2, 1200):
        for ni in set(orc.split(n)):
            for t in range(n):
                fl = orc.child_slope(n, ni, t)
                a, d = t * (ni - 1), n - 1
                q, r = divmod(a, d)
                exact = q + 1 if 2 * r > d else q if 2 * r < d else q + (q & 1)
                if fl != exact:
                    assert 2 * r == d, (n, ni, t)  # only at exact ties
                    assert abs(fl - exact) == 1
                    diffs += 1
                    first = first or n
    assert diffs > 0 and first == 23


def test_float_rule_recursion_equals_brute(orc_float):
    orc = orc_float
    rng = np.random.default_rng(3)
    for h, w in [(23, 5), (45, 7), (91, 3), (13, 11)]:
        img = rng.integers(0, 256, (h, w)).astype(np.int64)
        for b in (orc.CYCLIC, orc.EXTENDED):
            assert np.array_equal(orc.fht(img, 15, b), orc.brute(img, 15, b))
