"""Writes config4_coarse_gradient.txt: the dense FP64 oracle's energies and
adjoint gradients (dF/dq, dF/dsigma0, dF/dt) of the differentiation workload's
coarse version (tests/problems.py: config4_coarse).  Calls only the seeded
generators and oracle/; run from the repository root:
    python tests/golden/make_config4_coarse_gradient.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path[:0] = [ROOT, os.path.dirname(HERE)]

import numpy as np  # noqa: E402

from oracle.gradient import gradients  # noqa: E402
from problems import config4_coarse, oracle_system  # noqa: E402


def main():
    so = oracle_system(config4_coarse(), theta=0.0)
    g = gradients(so)
    e = g["energies"]
    out = os.path.join(HERE, "config4_coarse_gradient.txt")
    with open(out, "w") as fh:
        fh.write("# dense FP64 oracle (oracle.gradient.gradients), star molecule 2000 panels / 900 charges\n")
        fh.write("# 10 A from a 40 A sphere (3380 panels, sigma0 -0.05 C/m^2); kcal/mol, per e, per C/m^2, per A\n")
        for k in ("coulomb", "solvation", "surface", "total"):
            fh.write(f"energy {k} {e[k]:.17e}\n")
        fh.write(f"dbc 1 {g['dbc'][1]:.17e}\n")
        for b in range(2):
            fh.write("dt %d %s\n" % (b, " ".join(f"{v:.17e}" for v in g["dt"][b])))
        for k, v in enumerate(g["dq"][0]):
            fh.write(f"dq {k} {v:.17e}\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
