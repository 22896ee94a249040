"""Host side of the experiments module (CPU only).

``summary`` turns error numerators into Section 5's printed aggregates; fed
the oracle-written table of exact numerators for n = 1..4096 it must print the
paper's figures (36.38 % of n with the Theorem 2 bound below E_S, E_S / E_T
above 1.69 at n = 1451, E_T within Theorem 2 everywhere).  ``addition_counts``
reads Theorem 1's count from a host-only plan.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pattern_errors.txt")


@pytest.fixture(scope="module")
def table():
    return np.loadtxt(GOLDEN, dtype=np.int64)


def test_summary_prints_the_papers_aggregates(table):
    from paper_2411_07351_gb300.experiments import summary

    assert list(table[:, 0]) == list(range(1, 4097))
    s = summary([int(v) for v in table[:, 1]], [int(v) for v in table[:, 2]])
    assert round(s["share_bound_below_E_S_pct"], 2) == 36.38
    assert s["at_n"] == 1451 and 1.69 < s["max_E_S_over_E_T"] < 1.70
    assert s["E_T_within_theorem2"]


def test_summary_of_a_sub_range(table):
    from paper_2411_07351_gb300.experiments import summary

    # n = 1440..1460 holds the peak ratio; the share is of the sub-range only
    s = summary([int(v) for v in table[1439:1460, 1]], [int(v) for v in table[1439:1460, 2]], n_lo=1440)
    assert s["at_n"] == 1451
    assert 0.0 <= s["share_bound_below_E_S_pct"] <= 100.0


@pytest.mark.parametrize("n", [1, 2, 3, 17, 100, 1024, 4095])
def test_addition_counts_are_theorem_1(orc, n):
    from paper_2411_07351_gb300 import build as B

    B.build()
    from paper_2411_07351_gb300.experiments import addition_counts

    assert addition_counts(n, "T") == orc.adds(n, orc.SPLIT_T)
    assert addition_counts(n, "S") == orc.adds(n, orc.SPLIT_S)
