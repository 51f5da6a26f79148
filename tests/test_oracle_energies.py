"""Pins of the oracle's system, solve and energies against closed forms and
the analytical solution of Section 4."""
import math
import os

import numpy as np
import pytest
from scipy.special import eval_legendre, spherical_in, spherical_kn

import synth
from oracle import units
from oracle.analytical import (B_matrix, interaction, isolated_molecule_solvation,
                               isolated_surface_charge, isolated_surface_potential)
from oracle.bem import DIELECTRIC, SET_CHARGE, SET_POTENTIAL, Body, System
from oracle.energy import energies, interaction_energy

C_KCAL = 332.0637  # e^2/(4 pi eps0 A) in kcal/mol, textbook value


def test_units():
    assert units.COULOMB_KCAL == pytest.approx(C_KCAL, rel=2e-7)
    assert units.sigma_from_c_m2(0.05) == pytest.approx(3.1207545e-3, rel=1e-7)
    assert units.phi_from_volt(1.0) == pytest.approx(5.526350e-3, rel=1e-5)


def kirkwood(a, q, ein, eout, kappa):
    # Born ion in a salt solution (Kirkwood, single central charge)
    return 0.5 * q * q * units.COULOMB_KCAL * (1.0 / (eout * (1 + kappa * a)) - 1.0 / ein) / a


def test_isolated_limits_are_textbook_forms():
    s0 = units.sigma_from_c_m2(0.05)
    p0 = units.phi_from_volt(0.05)
    d, eps, k = 4.0, 80.0, 0.125
    # isolated sphere held at phi0:  F = -2 pi eps phi0^2 d (1 + kappa d)
    fp = -2 * math.pi * eps * p0 ** 2 * d * (1 + k * d) * units.ENERGY_KCAL
    # isolated sphere of charge sigma0: F = 2 pi sigma0^2 d^3 / (eps (1 + kappa d))
    fc = 2 * math.pi * s0 ** 2 * d ** 3 / (eps * (1 + k * d)) * units.ENERGY_KCAL
    assert isolated_surface_potential(d, p0, eps, k) == pytest.approx(fp, rel=1e-12)
    assert isolated_surface_charge(d, s0, eps, k) == pytest.approx(fc, rel=1e-12)
    assert fp == pytest.approx(-0.96088, abs=1e-5)
    assert fc == pytest.approx(0.136185, abs=1e-6)
    assert isolated_surface_charge(40.0, -s0, eps, k) == pytest.approx(34.046, abs=1e-3)
    assert isolated_molecule_solvation(4.0, 1.0, 4.0, 80.0, 0.125) == pytest.approx(
        kirkwood(4.0, 1.0, 4.0, 80.0, 0.125), rel=1e-12)
    assert kirkwood(4.0, 1.0, 4.0, 80.0, 0.125) == pytest.approx(-10.0311, abs=1e-4)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_addition_theorem(n):
    # k_n(kappa r2) P_n(cos th2) = sum_m (2m+1) B_nm i_m(kappa r1) P_m(cos th1), Eq. 19 (addition_formula),
    # each angle measured from the line of centres towards the other centre
    kappa, R = 0.125, 12.0
    B = B_matrix(50, kappa * R)
    rng = np.random.default_rng(n)
    for _ in range(5):
        r1 = rng.uniform(0.5, 5.0)
        th1 = rng.uniform(0, math.pi)
        p = np.array([r1 * math.sin(th1), 0.0, r1 * math.cos(th1)])   # centre 2 at +z R
        d2 = p - np.array([0, 0, R])
        r2 = np.linalg.norm(d2)
        cos2 = (-d2[2]) / r2       # angle from the axis pointing towards centre 1
        lhs = spherical_kn(n, kappa * r2) * eval_legendre(n, cos2)
        rhs = sum((2 * m + 1) * B[n, m] * spherical_in(m, kappa * r1) * eval_legendre(m, math.cos(th1))
                  for m in range(50))
        assert rhs == pytest.approx(lhs, rel=1e-9)


def test_analytical_series_converges_and_decays_with_distance():
    s0 = units.sigma_from_c_m2(0.05)
    e20 = interaction(4, 4, 12, 1, 4, 80, 0.125, sigma0=s0, N=20)[0]
    e40 = interaction(4, 4, 12, 1, 4, 80, 0.125, sigma0=s0, N=40)[0]
    assert e20 == pytest.approx(e40, rel=1e-9)
    far = interaction(4, 4, 400, 1, 4, 80, 0.125, sigma0=s0, N=20)[0]
    assert abs(far) < 1e-12
    B = B_matrix(12, 1.5)
    assert np.allclose(B, B.T, rtol=1e-13)


def _mol(level, r=4.0):
    v, f = synth.icosphere(level, r)
    return Body(DIELECTRIC, v, f, eps_in=4.0, charge_xyz=np.zeros((1, 3)), charge_q=np.array([1.0]))


def test_kirkwood_sphere_converges_at_first_order():
    exact = kirkwood(4.0, 1.0, 4.0, 80.0, 0.125)
    errs = []
    for level in (2, 3):
        s = System([_mol(level)], 80.0, 0.125)
        errs.append(energies(s, s.solve())["solvation"] - exact)
    ratio = errs[0] / errs[1]
    assert 3.3 < ratio < 4.7          # error ~ 1/N, N grows 4x per level
    rich = (4 * (exact + errs[1]) - (exact + errs[0])) / 3
    assert abs(rich - exact) < 2e-3


@pytest.mark.parametrize("kind", [SET_CHARGE, SET_POTENTIAL])
def test_two_sphere_interaction_converges_to_analytical(kind):
    s0 = units.sigma_from_c_m2(0.05)
    p0 = units.phi_from_volt(0.05)
    val = s0 if kind == SET_CHARGE else p0
    kw = {"sigma0": s0} if kind == SET_CHARGE else {"phi0": p0}
    ana = interaction(4, 4, 12, 1, 4, 80, 0.125, **kw)[0]
    errs = []
    for level in (2, 3):
        v, f = synth.icosphere(level, 4.0)
        mol = _mol(level)
        srf = Body(kind, v + np.array([12.0, 0, 0]), f, bc_value=val)
        s = System([mol, srf], 80, 0.125)
        tot = energies(s, s.solve())["total"]
        sm, ss = System([mol], 80, 0.125), System([srf], 80, 0.125)
        tm = energies(sm, sm.solve())["total"]
        ts = energies(ss, ss.solve())["total"]
        errs.append(interaction_energy(tot, [tm, ts]) - ana)
    assert 3.0 < errs[0] / errs[1] < 5.0
    assert abs(errs[1]) < 0.02 * abs(ana)


def test_matrix_free_rows_equal_dense_matrix():
    v, f = synth.icosphere(1, 4.0)
    mol = _mol(1)
    srf = Body(SET_POTENTIAL, v + np.array([9.0, 1.0, 0]), f, bc_value=0.01)
    s = System([mol, srf], 80, 0.125)
    A, _ = s.assemble()
    x = np.random.default_rng(3).normal(size=s.n)
    assert np.allclose(A @ x, s.apply(x), rtol=0, atol=1e-13)


def test_printed_interaction_energies_arithmetic():
    path = os.path.join(os.path.dirname(__file__), "golden", "printed_energies.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for name, iso_s, iso_f, int_s, int_f, printed, tol in rows:
        f = interaction_energy(float(int_s) + float(int_f), [float(iso_s) + float(iso_f)])
        assert abs(f - float(printed)) <= float(tol), name
