"""Write ``pattern_errors.txt``: the exact maximum orthotropic error of the
FHT2DS and FHT2DT generating patterns for every n in [1, 4096].

Section 5 of the paper evaluates E_S(n) and E_T(n) over all patterns of both
families for n <= 4096 and prints three aggregates of the result (the share of
n where the Theorem 2 bound lies strictly below E_S(n), the largest E_S/E_T
ratio and where it occurs, and the sizes of the highest E_S peaks).  The test
``tests/test_oracle_paper_aggregates.py`` checks this table against those
printed aggregates and re-derives a sample of its rows from the oracle.

This script calls only ``oracle``.  Columns: n, num_S, num_T, where
E(n) = num / (n - 1) (0 for n = 1).

Run:  python tests/golden/make_pattern_errors.py
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

N_MAX = 4096


def _row(n):
    return n, oracle.pattern_error_num(n, oracle.SPLIT_S), oracle.pattern_error_num(n, oracle.SPLIT_T)


def main():
    oracle.build()
    order = sorted(range(1, N_MAX + 1), reverse=True)  # largest first for load balance
    with mp.get_context("spawn").Pool() as pool:
        rows = sorted(pool.map(_row, order, chunksize=8))
    path = os.path.join(HERE, "pattern_errors.txt")
    with open(path, "w") as f:
        f.write("# Exact maximum orthotropic pattern error, Section 4-5 of arXiv 2411.07351.\n")
        f.write("# E(n) = num / (n - 1); written by tests/golden/make_pattern_errors.py from oracle/.\n")
        f.write("# n num_S num_T\n")
        for n, s, t in rows:
            f.write(f"{n} {s} {t}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
