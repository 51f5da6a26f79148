"""Derive the triangle and edge quadrature rules used by the CUDA library and
write them to csrc/pgb_rules.h.

Section 3.1 of the paper integrates far panels with 1, 3, 4 or 7 Gauss
points, panels closer than 2L with 19 points (37 in Table 1) and the self
panel with Gauss points along its edges, without printing the rules.  This
library uses the fully symmetric rules of degree 1, 2, 3, 5, 9 and 13 with the
fewest orbits.
Each is found here by Newton's method on its moment equations (the exact
integrals of x^i y^j over the unit right triangle, normalised to unit area),
starting from a rough guess; the edge rule is Gauss-Legendre on [0, 1],
computed by Newton iteration on the Legendre recurrence.

Run:  python -m paper_1506_03745_gb300.gen_rules   (rewrites the header)
"""
import math
import os

import numpy as np

# (degree, orbits) with orbit kinds 'c' centroid (w), 'a' (w, a) for the
# barycentric point (a, a, 1-2a) and its rotations, 'b' (w, a, b) for the six
# permutations of (a, b, 1-a-b); rough starting values.
SPECS = {
    1: (1, [("c", [1.0])]),
    3: (2, [("a", [0.3, 0.2])]),
    4: (3, [("c", [-0.6]), ("a", [0.5, 0.21])]),
    7: (5, [("c", [0.2]), ("a", [0.12, 0.46]), ("a", [0.14, 0.11])]),
    19: (9, [("c", [0.1]), ("a", [0.03, 0.49]), ("a", [0.08, 0.44]),
             ("a", [0.08, 0.19]), ("a", [0.025, 0.045]), ("b", [0.045, 0.035, 0.22])]),
    # degree 13 with 21 parameters: the count of fully symmetric moment
    # conditions of degree <= 13 (one per e2^a e3^b with 2a + 3b <= 13)
    37: (13, [("c", [0.07]), ("a", [0.06, 0.22]), ("a", [0.024, 0.49]), ("a", [0.006, 0.022]),
              ("a", [0.055, 0.43]), ("b", [0.015, 0.024, 0.86]), ("b", [0.0096, 0.27, 0.72]),
              ("b", [0.035, 0.07, 0.62]), ("b", [0.024, 0.16, 0.75])]),
}
# rules solved for relative moment errors (each equation divided by its exact
# moment): the degree-13 moments span many orders of magnitude
RELATIVE = {37}
EDGE_POINTS = (3, 6, 9, 12)


def points(params, orbits):
    bary, wts = [], []
    i = 0
    for kind, _ in orbits:
        if kind == "c":
            bary.append((1 / 3, 1 / 3, 1 / 3))
            wts.append(params[i])
            i += 1
        elif kind == "a":
            w, a = params[i:i + 2]
            i += 2
            for t in ((a, a, 1 - 2 * a), (a, 1 - 2 * a, a), (1 - 2 * a, a, a)):
                bary.append(t)
                wts.append(w)
        else:
            w, a, b = params[i:i + 3]
            i += 3
            c = 1 - a - b
            for t in ((a, b, c), (b, a, c), (a, c, b), (c, a, b), (b, c, a), (c, b, a)):
                bary.append(t)
                wts.append(w)
    return np.array(bary), np.array(wts)


def residual(params, orbits, degree, relative=False):
    bary, w = points(params, orbits)
    out = []
    for i in range(degree + 1):
        for j in range(degree + 1 - i):
            exact = 2.0 * math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            r = np.dot(w, bary[:, 0] ** i * bary[:, 1] ** j) - exact
            out.append(r / exact if relative else r)
    return np.array(out)


def newton(orbits, degree, x0, iters=60, relative=False):
    """Gauss-Newton with a complex-step Jacobian (exact to rounding)."""
    x = np.array(x0, dtype=np.float64)
    for _ in range(iters):
        f = residual(x, orbits, degree, relative).real
        J = np.empty((len(f), len(x)))
        for k in range(len(x)):
            e = np.zeros(len(x), dtype=np.complex128)
            e[k] = 1e-30j
            J[:, k] = residual(x + e, orbits, degree, relative).imag / 1e-30
        step = np.linalg.lstsq(J, -f, rcond=None)[0]
        x = x + step
        if np.max(np.abs(step)) < 1e-17:
            break
    if np.max(np.abs(residual(x, orbits, degree).real)) > 1e-15:
        raise RuntimeError("moment equations not solved")
    return x


def triangle_rule(K):
    degree, orbits = SPECS[K]
    x0 = [v for _, vals in orbits for v in vals]
    x = np.array([1.0]) if K == 1 else newton(orbits, degree, x0, iters=200 if K in RELATIVE else 60,
                                              relative=K in RELATIVE)
    bary, w = points(x, orbits)
    return np.real(bary) - 1.0 / 3.0, np.real(w)


def gauss_legendre01(n):
    """Nodes/weights on [0,1]: roots of P_n by Newton on the three-term recurrence."""
    xs, ws = [], []
    for i in range(1, n + 1):
        x = math.cos(math.pi * (i - 0.25) / (n + 0.5))
        for _ in range(100):
            p0, p1 = 1.0, x
            for k in range(2, n + 1):
                p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
            dp = n * (x * p1 - p0) / (x * x - 1.0)
            dx = p1 / dp
            x -= dx
            if abs(dx) < 1e-17:
                break
        p0, p1 = 1.0, x
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        xs.append(0.5 * (1.0 - x))
        ws.append(1.0 / ((1.0 - x * x) * dp * dp))
    order = np.argsort(xs)
    return np.array(xs)[order], np.array(ws)[order]


def header():
    lines = ["// Generated by paper_1506_03745_gb300/gen_rules.py -- do not edit.",
             "// Symmetric triangle rules (barycentric offsets mu = lambda - 1/3 from the",
             "// centroid, weights summing to one) and Gauss-Legendre rules on [0,1].",
             "#pragma once", ""]
    for K in sorted(SPECS):
        mu, w = triangle_rule(K)
        mu[np.all(np.abs(mu) < 1e-15, axis=1)] = 0.0
        lines.append(f"static const double PGB_TRI{K}_MU[{K}][3] = {{")
        lines += ["    {%.17e, %.17e, %.17e}," % tuple(m) for m in mu]
        lines.append("};")
        lines.append(f"static const double PGB_TRI{K}_W[{K}] = {{")
        lines += ["    %.17e," % v for v in w]
        lines.append("};")
        lines.append("")
    for n in EDGE_POINTS:
        x, w = gauss_legendre01(n)
        lines.append(f"static const double PGB_GL{n}_X[{n}] = {{" + ", ".join("%.17e" % v for v in x) + "};")
        lines.append(f"static const double PGB_GL{n}_W[{n}] = {{" + ", ".join("%.17e" % v for v in w) + "};")
    return "\n".join(lines) + "\n"


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "pgb_rules.h")
    with open(path, "w") as f:
        f.write(header())
    print("wrote", path)


if __name__ == "__main__":
    main()
