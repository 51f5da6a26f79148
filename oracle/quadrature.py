"""Quadrature rules for flat triangular panels (Section 3.1).

The paper integrates far panels with 1, 3, 4 or 7 Gauss points, close panels
(closer than 2L) with a rule of 19 or more points, and the panel that holds the
collocation point semi-analytically with Gauss points along its edges.  It does
not print the rules.  The oracle's reading: fully symmetric rules with the
fewest orbits that reach the degrees 1 (K=1), 2 (K=3), 3 (K=4), 5 (K=7) and
9 (K=19), and for the 37-point close-by rule of Table 1 the fully symmetric
rule of degree 13 whose orbit count matches its moment conditions.  Each rule is *derived here* by solving its moment equations
sum_m w_m x_m^i y_m^j = 2 i! j!/(i+j+2)!  (exact monomial integrals over the
reference triangle, normalised to unit area) for the weights and orbit
parameters, from a rough starting point, with Levenberg-Marquardt.

A rule is returned as (mu (K,3), w (K,)): mu_a = lambda_a - 1/3 are barycentric
offsets from the centroid (the centroid node has mu = 0 exactly) and the
weights sum to one (fractions of the panel area).
"""
from functools import lru_cache
from math import factorial

import numpy as np
from scipy.optimize import least_squares

# orbit structure and a rough (2-digit) starting point for each rule:
# 'c' = centroid (w), 'a' = S21 orbit (w, a) with barycentric (a, a, 1-2a),
# 'b' = S111 orbit (w, a, b) with barycentric permutations of (a, b, 1-a-b).
_RULES = {
    1: (1, [("c", (1.0,))]),
    3: (2, [("a", (0.33, 0.17))]),
    4: (3, [("c", (-0.5,)), ("a", (0.5, 0.2))]),
    7: (5, [("c", (0.22,)), ("a", (0.13, 0.47)), ("a", (0.13, 0.10))]),
    19: (9, [("c", (0.097,)), ("a", (0.031, 0.49)), ("a", (0.078, 0.44)),
             ("a", (0.080, 0.19)), ("a", (0.026, 0.045)), ("b", (0.043, 0.037, 0.22))]),
    # degree 13: the fully symmetric moment conditions up to degree 13 are
    # 21 (the symmetric polynomials e2^a e3^b, 2a + 3b <= 13), met by the
    # centroid, four 3-point and four 6-point orbits (21 unknowns, 37 points)
    37: (13, [("c", (0.068,)), ("a", (0.058, 0.22)), ("a", (0.024, 0.49)), ("a", (0.0061, 0.022)),
              ("a", (0.056, 0.43)), ("b", (0.015, 0.024, 0.86)), ("b", (0.0096, 0.27, 0.72)),
              ("b", (0.035, 0.068, 0.62)), ("b", (0.024, 0.16, 0.75))]),
}
# rules whose moment equations are solved relative to the exact moments: the
# degree-13 moments span many orders of magnitude, and unscaled equations leave
# the orbit parameters undetermined beyond about 1e-6
_RELATIVE = {37}


def _expand(params, struct):
    lam, w = [], []
    k = 0
    for kind, _ in struct:
        if kind == "c":
            lam.append((1 / 3, 1 / 3, 1 / 3)); w.append(params[k]); k += 1
        elif kind == "a":
            wt, a = params[k], params[k + 1]; k += 2
            for p in ((a, a, 1 - 2 * a), (a, 1 - 2 * a, a), (1 - 2 * a, a, a)):
                lam.append(p); w.append(wt)
        else:
            wt, a, b = params[k], params[k + 1], params[k + 2]; k += 3
            c = 1 - a - b
            for p in ((a, b, c), (b, a, c), (a, c, b), (c, a, b), (b, c, a), (c, b, a)):
                lam.append(p); w.append(wt)
    return np.array(lam), np.array(w)


def _moment_residual(params, struct, deg, relative=False):
    lam, w = _expand(params, struct)
    x, y = lam[:, 0], lam[:, 1]
    res = []
    for i in range(deg + 1):
        for j in range(deg + 1 - i):
            exact = 2.0 * factorial(i) * factorial(j) / factorial(i + j + 2)
            r = np.sum(w * x ** i * y ** j) - exact
            res.append(r / exact if relative else r)
    return np.array(res)


@lru_cache(maxsize=None)
def triangle_rule(K: int):
    """Symmetric K-point rule on a triangle, as (mu, w); see the module doc."""
    if K not in _RULES:
        raise ValueError(f"no {K}-point triangle rule")
    deg, struct = _RULES[K]
    x0 = np.concatenate([np.asarray(p, dtype=np.float64) for _, p in struct])
    if K == 1:
        params = np.array([1.0])
    else:
        sol = least_squares(_moment_residual, x0, args=(struct, deg, K in _RELATIVE), method="lm",
                            xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
        params = sol.x
    lam, w = _expand(params, struct)
    mu = lam - 1.0 / 3.0
    # the centroid node is exactly mu = 0
    mu[np.all(np.abs(mu) < 1e-14, axis=1)] = 0.0
    return mu, w


def rule_degree(K: int) -> int:
    return _RULES[K][0]


@lru_cache(maxsize=None)
def gauss_legendre01(n: int):
    """n-point Gauss-Legendre rule on [0, 1] (nodes, weights)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w
