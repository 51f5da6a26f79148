"""Pins of the oracle's panel integrals and operators (Section 3.1, Eq. 8-9)."""
import math

import numpy as np
import pytest
from scipy import integrate

import synth
from oracle.geometry import Panels
from oracle.integrals import panel_operator_blocks, self_integral


def _tri():
    return np.array([[0.0, 0.0, 0.0], [1.3, 0.1, 0.0], [0.2, 0.9, 0.0]])


def test_laplace_self_integral_matches_closed_form():
    # int_subtriangle 1/(4 pi r) dA about the apex = h/(4 pi) [asinh(s/h)]_{s_a}^{s_b}
    v = _tri()
    c = v.mean(0)
    exact = 0.0
    for a in range(3):
        pa, pb = v[a], v[(a + 1) % 3]
        u = (pb - pa) / np.linalg.norm(pb - pa)
        foot = pa + ((c - pa) @ u) * u
        h = np.linalg.norm(c - foot)
        sa, sb = (pa - foot) @ u, (pb - foot) @ u
        exact += h / (4 * math.pi) * (math.asinh(sb / h) - math.asinh(sa / h))
    # the edge rule converges to the closed form; 9 points per edge (the
    # paper's setting) is within 1e-3 for this skewed panel
    VL40, _ = self_integral(v, c, 0.0, 40)
    assert abs(VL40 - exact) / exact < 1e-11
    VL, VY = self_integral(v, c, 0.0, 9)
    assert abs(VL - exact) / exact < 1e-3
    assert VY == pytest.approx(VL, rel=1e-15)


def test_yukawa_self_integral_matches_adaptive_quadrature():
    v = _tri()
    c = v.mean(0)
    kappa = 0.7
    # polar coordinates about c, radial integral numerically (independent of the
    # closed-form radial step of the semi-analytical rule)
    total = 0.0
    for a in range(3):
        pa, pb = v[a] - c, v[(a + 1) % 3] - c
        th_a, th_b = math.atan2(pa[1], pa[0]), math.atan2(pb[1], pb[0])
        if th_b < th_a:
            th_b += 2 * math.pi
        e = pb - pa

        def rho(th):
            d = np.array([math.cos(th), math.sin(th), 0.0])
            # intersect ray c + t d with edge pa + s e
            M = np.array([[d[0], -e[0]], [d[1], -e[1]]])
            t, _ = np.linalg.solve(M, pa[:2])
            return t

        val, _ = integrate.dblquad(lambda r, th: math.exp(-kappa * r) / (4 * math.pi),
                                   th_a, th_b, lambda th: 0.0, rho, epsabs=1e-13, epsrel=1e-12)
        total += val
    _, VY = self_integral(v, c, kappa, 40)
    assert abs(VY - total) / total < 1e-10
    _, VY9 = self_integral(v, c, kappa, 9)
    assert abs(VY9 - total) / total < 1e-3


def _sphere_rowsums(level, a=2.0, kappa=0.3):
    v, f = synth.icosphere(level, a)
    p = Panels(v, f)
    VL, KL, VY, KY = panel_operator_blocks(p.c, p, kappa, 7, 19, 9, np.arange(p.N))
    return p, VL.sum(1), KL.sum(1), VY.sum(1), KY.sum(1)


def test_sphere_row_sum_identities_converge():
    # exact continuum row sums for a sphere of radius a with the collocation
    # point on it (dA = 2 pi r dr over the chord length r in [0, 2a]):
    a, kappa = 2.0, 0.3
    e2 = math.exp(-2 * kappa * a)
    exact = dict(VL=a, KL=-0.5, VY=(1 - e2) / (2 * kappa),
                 KY=-(1 - e2) / (2 * kappa * a) + e2 / 2)
    errs = []
    for level in (2, 3):
        _, vl, kl, vy, ky = _sphere_rowsums(level, a, kappa)
        errs.append({k: np.abs(s - exact[k]).max() for k, s in zip(("VL", "KL", "VY", "KY"), (vl, kl, vy, ky))})
    for k in ("VL", "VY", "KY"):
        assert errs[1][k] < errs[0][k] / 2.5, (k, errs)
        assert errs[1][k] < 0.02 * abs(exact[k]) + 2e-3
    # Gauss's law: at a point on a face of a closed polyhedron the Laplace
    # double layer of a unit density is exactly -1/2; what remains is the
    # error of the 7- and 19-point rules
    assert errs[0]["KL"] < 5e-4 and errs[1]["KL"] < 5e-4


def test_tier_switch_is_continuous_to_rule_accuracy():
    # just outside 2L the K-point value and the fine value agree closely
    v, f = synth.icosphere(2, 3.0)
    p = Panels(v, f)
    j = 0
    x = p.c[j] + p.n[j] * (2.0 * p.L[j] + 1e-9)
    far = panel_operator_blocks(x[None], p, 0.2, 7, 19, 9, None)
    near = panel_operator_blocks(x[None], p, 0.2, 19, 19, 9, None)
    for a, b in zip(far, near):
        assert abs(a[0, j] - b[0, j]) < 1e-3 * abs(b[0, j]) + 1e-12
