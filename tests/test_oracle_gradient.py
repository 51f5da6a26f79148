"""Pins of the dense adjoint gradients (oracle/gradient.py): central finite
differences, Euler's identity for a quadratic form, translation invariance."""
import numpy as np
import pytest

import synth
from oracle import units
from oracle.bem import DIELECTRIC, SET_CHARGE, SET_POTENTIAL, Body, System
from oracle.energy import energies
from oracle.gradient import gradients


def _system(kind=SET_CHARGE, q=None, t=(9.5, 0.4, -0.3), bc=None, level=1):
    v, f = synth.star_surface(4, 3, 3.0)
    rng = np.random.default_rng(2)
    xyz = rng.uniform(-0.8, 0.8, size=(4, 3))
    q = rng.uniform(-1, 1, 4) if q is None else q
    mol = Body(DIELECTRIC, v, f, eps_in=4.0, charge_xyz=xyz, charge_q=q)
    v2, f2 = synth.icosphere(level, 3.0)
    if bc is None:
        bc = units.sigma_from_c_m2(-0.05) if kind == SET_CHARGE else units.phi_from_volt(0.05)
    srf = Body(kind, v2, f2, bc_value=bc, t=np.asarray(t, dtype=float))
    return System([mol, srf], 80.0, 0.125)


def _total(sys):
    return energies(sys, sys.solve())["total"]


@pytest.mark.parametrize("kind", [SET_CHARGE, SET_POTENTIAL])
def test_charge_gradient_matches_finite_differences(kind):
    s = _system(kind)
    gr = gradients(s)
    q0 = s.bodies[0].charge_q.copy()
    for k in (0, 3):
        h = 1e-4
        s.bodies[0].charge_q = q0.copy(); s.bodies[0].charge_q[k] += h
        fp = _total(s)
        s.bodies[0].charge_q = q0.copy(); s.bodies[0].charge_q[k] -= h
        fm = _total(s)
        s.bodies[0].charge_q = q0
        assert gr["dq"][0][k] == pytest.approx((fp - fm) / (2 * h), rel=1e-6)


@pytest.mark.parametrize("kind", [SET_CHARGE, SET_POTENTIAL])
def test_translation_gradient_matches_finite_differences(kind):
    t0 = np.array([9.5, 0.4, -0.3])
    gr = gradients(_system(kind, t=t0))
    h = 1e-3
    for ax in range(3):
        tp = t0.copy(); tp[ax] += h
        tm = t0.copy(); tm[ax] -= h
        fd = (_total(_system(kind, t=tp)) - _total(_system(kind, t=tm))) / (2 * h)
        # moving the surface by +h is moving the molecule by -h
        assert gr["dt"][1][ax] == pytest.approx(fd, rel=1e-4, abs=1e-9)
    np.testing.assert_allclose(gr["dt"][0], -gr["dt"][1], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("kind", [SET_CHARGE, SET_POTENTIAL])
def test_bc_gradient_and_euler_identity(kind):
    s = _system(kind)
    gr = gradients(s)
    bc = s.bodies[1].bc_value
    conv = units.sigma_from_c_m2(1.0) if kind == SET_CHARGE else units.phi_from_volt(1.0)
    h = 1e-3 * abs(bc)
    fp = _total(_system(kind, bc=bc + h))
    fm = _total(_system(kind, bc=bc - h))
    assert gr["dbc"][1] == pytest.approx((fp - fm) / (2 * h) * conv, rel=1e-6)
    # F is a homogeneous quadratic form in (q, bc): q.dF/dq + bc dF/dbc = 2F
    lhs = s.bodies[0].charge_q @ gr["dq"][0] + (bc / conv) * gr["dbc"][1]
    assert lhs == pytest.approx(2 * gr["energies"]["total"], rel=1e-10)
