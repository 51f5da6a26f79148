"""Pins of the oracle's triangle and edge rules (Section 3.1)."""
import math
from math import factorial

import numpy as np
import pytest

from oracle.quadrature import gauss_legendre01, rule_degree, triangle_rule


@pytest.mark.parametrize("K", [1, 3, 4, 7, 19, 37])
def test_rule_integrates_monomials_to_its_degree(K):
    mu, w = triangle_rule(K)
    lam = mu + 1.0 / 3.0
    x, y = lam[:, 0], lam[:, 1]
    deg = rule_degree(K)
    for i in range(deg + 1):
        for j in range(deg + 1 - i):
            exact = 2.0 * factorial(i) * factorial(j) / factorial(i + j + 2)
            assert abs(np.sum(w * x ** i * y ** j) - exact) < 1e-14
    # and fails one degree higher (the degree is sharp), except for K=1 whose
    # centroid rule is also exact for the degree-1 monomials only
    # (relative to the exact moment: the degree-14 moments are small)
    errs = []
    for i in range(deg + 2):
        exact = 2.0 * factorial(i) * factorial(deg + 1 - i) / factorial(deg + 3)
        errs.append(abs(np.sum(w * x ** i * y ** (deg + 1 - i)) - exact) / exact)
    assert max(errs) > 1e-5
    assert np.all(lam > 0) and np.all(lam < 1)
    assert abs(w.sum() - 1.0) < 1e-15


def test_seven_point_rule_is_radons_closed_form():
    # Radon's degree-5 rule: centroid weight 9/40, orbits a = (6 -+ sqrt15)/21
    # with weights (155 -+ sqrt15)/1200 (textbook closed form, independent of
    # the moment solver).
    mu, w = triangle_rule(7)
    lam = np.sort(mu + 1.0 / 3.0, axis=1)
    s15 = math.sqrt(15.0)
    expect = {round(9 / 40, 12): (1 / 3,),
              round((155 - s15) / 1200, 12): ((6 - s15) / 21,),
              round((155 + s15) / 1200, 12): ((6 + s15) / 21,)}
    for lw, l in zip(w, lam):
        key = round(lw, 12)
        assert key in expect
        a = expect[key][0]
        assert abs(l[0] - a) < 1e-13 or abs(l[1] - a) < 1e-13


def test_four_point_rule_closed_form():
    mu, w = triangle_rule(4)
    assert abs(w[0] + 27.0 / 48.0) < 1e-13
    assert np.allclose(w[1:], 25.0 / 48.0, atol=1e-13)
    assert np.allclose(np.sort(mu[1] + 1 / 3), [0.2, 0.2, 0.6], atol=1e-13)


def test_gauss_legendre_edge_rule():
    x, w = gauss_legendre01(9)
    for p in range(18):
        assert abs(np.sum(w * x ** p) - 1.0 / (p + 1)) < 1e-14


def test_37_point_rule_is_fully_symmetric_and_beats_19_points():
    """The 37-point rule of Table 1 (degree 13): its nodes come in the orbits
    of the triangle's symmetry group (1 + 4 x 3 + 4 x 6), and on a smooth
    integrand with a closed-form integral, exp(x + 2y) over the reference
    triangle, its error is far below the 19-point rule's."""
    mu, w = triangle_rule(37)
    lam = mu + 1.0 / 3.0
    keys = {}
    for l, wt in zip(lam, w):
        k = (tuple(np.round(np.sort(l), 12)), round(wt, 13))
        keys[k] = keys.get(k, 0) + 1
    assert sorted(keys.values()) == [1] + [3] * 4 + [6] * 4
    # int over {x, y >= 0, x + y <= 1} of e^(x + 2y), normalised by the area 1/2:
    # inner integral over y then x gives (e^2 - 2e + 1) / 2, doubled
    exact = (math.e ** 2 - 2 * math.e + 1)

    def rule_err(K):
        m, wt = triangle_rule(K)
        lm = m + 1.0 / 3.0
        return abs(np.sum(wt * np.exp(lm[:, 0] + 2 * lm[:, 1])) - exact)

    assert rule_err(37) < 1e-13
    assert rule_err(37) < 1e-3 * rule_err(19)
