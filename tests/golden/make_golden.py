"""Writes the oracle-generated golden files of this folder.

It calls only the oracle (``oracle/``) and the seeded input generators
(``workloads/``); the stored values are therefore a regression pin of the
oracle on the 1,000 + 1,000-row, 4 + 4-column FP64 workload (100 keys).
Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from workloads import config  # noqa: E402


def main():
    A, B = config("c0")
    R, s = oracle.join_r_sigma(A.x, A.key, B.x, B.key, route="materialized")
    rows = oracle.join_rows(A.key, B.key)
    with open(os.path.join(HERE, "c0_oracle_R_sigma.txt"), "w") as f:
        f.write("# Oracle O1 (materialised join, Householder QR, one-sided Jacobi) on the\n")
        f.write("# seeded 1000+1000-row, 4+4-column FP64 workload with 100 keys.\n")
        f.write("# Written by tests/golden/make_golden.py (calls only oracle/ and workloads/).\n")
        f.write(f"join_rows {rows}\n")
        f.write("R " + " ".join(repr(float(v)) for v in R.ravel()) + "\n")
        f.write("sigma " + " ".join(repr(float(v)) for v in s) + "\n")


if __name__ == "__main__":
    main()
