"""Pins of the oracle treecode (Section 3.2): exact limit theta -> 0,
convergence in P, and the truncated kernels against independent closed forms."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre, spherical_kn

import synth
from oracle.bem import DIELECTRIC, SET_CHARGE, Body, Params, System
from oracle.treecode import TreecodeOperator, truncated_kernel


def _pair(seed):
    rng = np.random.default_rng(seed)
    R = rng.normal(size=(1, 3)) * 3
    d = rng.normal(size=(1, 3))
    d *= 0.45 * np.linalg.norm(R) / np.linalg.norm(d)
    return R, d, rng.normal(size=(1, 3))


@pytest.mark.parametrize("P", [0, 1, 3, 6])
def test_laplace_truncation_is_the_legendre_partial_sum(P):
    # 1/|R-d| = sum_n |d|^n / |R|^(n+1) P_n(cos g): the degree-n term is the
    # homogeneous degree-n part, so the degree-<=P truncations coincide
    R, d, p = _pair(P)
    F, _ = truncated_kernel(R, d, p, 0.0, P, True)
    r, dn = np.linalg.norm(R), np.linalg.norm(d)
    cg = float((R @ d.T).item()) / (r * dn)
    leg = sum(dn ** n / r ** (n + 1) * eval_legendre(n, cg) for n in range(P + 1)) / (4 * math.pi)
    assert F.item() == pytest.approx(leg, rel=1e-13)


def _double_factorial(n):
    return math.prod(range(n, 0, -2)) if n > 0 else 1


@pytest.mark.parametrize("P", [0, 2, 5, 7])
def test_yukawa_truncation_matches_gegenbauer_regrouping(P):
    # exp(-k|R-d|)/|R-d| = (2k/pi) sum_n (2n+1) i_n(k|d|) k_n(k|R|) P_n(cos g),
    # i_n(x) = x^n sum_j x^(2j) / (2^j j! (2n+2j+1)!!): collect total degree n+2j <= P
    kappa = 0.4
    R, d, p = _pair(10 + P)
    F, _ = truncated_kernel(R, d, p, kappa, P, False)
    r, dn = np.linalg.norm(R), np.linalg.norm(d)
    cg = float((R @ d.T).item()) / (r * dn)
    tot = 0.0
    for n in range(P + 1):
        for j in range((P - n) // 2 + 1):
            tot += ((2 * kappa / math.pi) * (2 * n + 1) * spherical_kn(n, kappa * r) * eval_legendre(n, cg)
                    * (kappa * dn) ** (n + 2 * j) / (2 ** j * math.factorial(j) * _double_factorial(2 * n + 2 * j + 1)))
    assert F.item() == pytest.approx(tot / (4 * math.pi), rel=1e-12)


@pytest.mark.parametrize("laplace", [True, False])
def test_double_layer_part_is_the_directional_derivative(laplace):
    R, d, p = _pair(5)
    h = 1e-5
    _, dF = truncated_kernel(R, d, p, 0.3, 5, laplace)
    Fp, _ = truncated_kernel(R, d + h * p, p, 0.3, 5, laplace)
    Fm, _ = truncated_kernel(R, d - h * p, p, 0.3, 5, laplace)
    assert dF.item() == pytest.approx((Fp - Fm).item() / (2 * h), rel=1e-7)


def _two_bodies():
    v, f = synth.icosphere(1, 4.0)
    v2, f2 = synth.icosphere(1, 3.0)
    mol = Body(DIELECTRIC, v, f, eps_in=4.0, charge_xyz=np.zeros((1, 3)), charge_q=np.array([1.0]))
    srf = Body(SET_CHARGE, v2 + np.array([8.5, 0.5, 0]), f2, bc_value=0.003)
    return System([mol, srf], 80.0, 0.125, Params(leaf_size=8, group_size=32))


def test_theta_zero_is_the_direct_sum():
    s = _two_bodies()
    x = np.random.default_rng(0).normal(size=s.n)
    y = TreecodeOperator(s, theta=0.0, P=3).apply(x)
    assert np.abs(y - s.apply(x)).max() < 1e-13


def test_error_decreases_with_order():
    s = _two_bodies()
    x = np.random.default_rng(1).normal(size=s.n)
    ref = s.apply(x)
    errs = []
    for P in (2, 6, 10):
        tc = TreecodeOperator(s, theta=0.5, P=P)
        assert sum(len(v[1]) for v in tc.lists.values()) > 0
        errs.append(np.abs(tc.apply(x) - ref).max() / np.abs(ref).max())
    assert errs[0] > 3 * errs[1] > 9 * errs[2]
