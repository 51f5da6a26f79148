"""Writes fullsize_rows.txt: rows of the oracle's treecode product (FP64,
oracle/treecode.py restricted to eight target groups) on the benchmark's
two-sphere workload at full size (2 x 20480 panels; theta 0.5, P 6, leaf 32,
K 7), for two seeded density vectors: positive densities (rows without
cancellation: compared row by row) and normal densities.  Calls only the
seeded generators and oracle/; run from the repository root:
    python tests/golden/make_fullsize_rows.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path[:0] = [ROOT, os.path.dirname(HERE)]

import numpy as np  # noqa: E402

from oracle.treecode import TreecodeOperator  # noqa: E402
from problems import fullsize_bodies, fullsize_groups, fullsize_vectors, oracle_system  # noqa: E402


def main():
    so = oracle_system(fullsize_bodies(), theta=0.5, P=6, leaf_size=32)
    tc = TreecodeOperator(so, groups=fullsize_groups())
    out = os.path.join(HERE, "fullsize_rows.txt")
    with open(out, "w") as fh:
        fh.write("# oracle treecode rows (theta 0.5, P 6, leaf 32, K 7), two spheres of 20480 panels\n")
        fh.write("# vector row value\n")
        for name, x in fullsize_vectors(so.n).items():
            y = tc.apply(x)
            for i in np.nonzero(np.isfinite(y))[0]:
                fh.write(f"{name} {i} {y[i]:.17e}\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
