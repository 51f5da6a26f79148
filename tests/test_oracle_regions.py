"""Pins of the oracle's multi-interface rows (oracle/regions.py): they reduce
to Eq. 6/7 without nesting, reproduce closed forms for a Stern layer and a
solvent-filled cavity, and leave the solution unchanged across an interface
with the same medium on both sides."""
import numpy as np
import pytest

import synth
from oracle import units
from oracle.bem import DIELECTRIC, SET_CHARGE, SET_POTENTIAL, Body, Params, System
from oracle.regions import RegionSystem, concentric_cavity_solvation, stern_sphere_solvation


def _mol(level, r, q=1.0, at=(0.0, 0.0, 0.0), eps_in=4.0):
    v, f = synth.icosphere(level, r)
    return Body(DIELECTRIC, v, f, eps_in=eps_in, charge_xyz=np.array([at], float), charge_q=np.array([q]))


def _shell(level, r, eps_in):
    v, f = synth.icosphere(level, r)
    return Body(DIELECTRIC, v, f, eps_in=eps_in)


def _energy(bodies, kappa, parent=None, kappa_in=None):
    rs = RegionSystem(bodies, 80.0, kappa, parent=parent, kappa_in=kappa_in, params=Params())
    return rs.energies(rs.solve())


@pytest.mark.parametrize("kind", [SET_CHARGE, SET_POTENTIAL, DIELECTRIC])
def test_rows_reduce_to_eq6_eq7_without_nesting(kind):
    v1, f1 = synth.icosphere(1, 4.0)
    v2, f2 = synth.icosphere(1, 3.0)
    b1 = Body(DIELECTRIC, v1, f1, eps_in=4.0, charge_xyz=np.array([[0.3, 0.0, 0.1]]), charge_q=np.array([1.0]))
    if kind == DIELECTRIC:
        b2 = Body(DIELECTRIC, v2 + [9.0, 0, 0], f2, eps_in=2.0, charge_xyz=np.array([[9.0, 0.2, 0.0]]),
                  charge_q=np.array([-0.5]))
    else:
        bc = units.sigma_from_c_m2(0.05) if kind == SET_CHARGE else units.phi_from_volt(0.05)
        b2 = Body(kind, v2 + [9.0, 0, 0], f2, bc_value=bc)
    A0, r0 = System([b1, b2], 80.0, 0.125).assemble()
    A1, r1 = RegionSystem([b1, b2], 80.0, 0.125).assemble()
    assert np.abs(A1 - A0).max() <= 1e-14 * np.abs(A0).max()
    assert np.abs(r1 - r0).max() <= 1e-14 * np.abs(r0).max()


def test_stern_layer_salt_term_matches_closed_form():
    """Central charge in a sphere of radius 4 inside an ion-free shell to
    radius 6: the salt-dependent part of the solvation energy, E(kappa) -
    E(0), is -q^2 kappa / (8 pi eps_out (1 + kappa b)) (the Born part
    cancels between the two solves on the same meshes).  Without the shell
    it would be 25 % larger in magnitude."""
    kap = 0.5
    m, s = _mol(3, 4.0), _shell(3, 6.0, 80.0)
    e_k = _energy([m, s], kap, parent=[1, -1])["solvation"]
    e_0 = _energy([m, s], 0.0, parent=[1, -1])["solvation"]
    exact = stern_sphere_solvation(1.0, 4.0, 6.0, 4.0, 80.0, kap) - stern_sphere_solvation(1.0, 4.0, 6.0, 4.0, 80.0, 0.0)
    no_shell = stern_sphere_solvation(1.0, 4.0, 4.0, 4.0, 80.0, kap) - stern_sphere_solvation(1.0, 4.0, 4.0, 4.0, 80.0, 0.0)
    assert (e_k - e_0) == pytest.approx(exact, rel=0.03)
    assert abs(no_shell - exact) > 0.2 * abs(exact)
    # the total solvation energy as well, at the mesh's discretisation error
    assert e_k == pytest.approx(stern_sphere_solvation(1.0, 4.0, 6.0, 4.0, 80.0, kap), rel=0.02)


def test_cavity_matches_series():
    """Charge 4 A from the centre of a sphere of radius 6 (eps 4) that holds a
    concentric cavity of radius 2: solvent-filled (eps 80) and, as a check of
    the rows alone, with the molecule's own permittivity (no effect)."""
    kap = 0.125
    out = {}
    for eps_c in (80.0, 4.0):
        m = _mol(3, 6.0, at=(4.0, 0.0, 0.0))
        c = _shell(3, 2.0, eps_c)
        out[eps_c] = _energy([m, c], kap, parent=[-1, 0])["solvation"]
        ref = concentric_cavity_solvation(1.0, 4.0, 2.0, 6.0, eps_c, 4.0, 80.0, kap)
        assert out[eps_c] == pytest.approx(ref, rel=0.02)
    d_ref = (concentric_cavity_solvation(1.0, 4.0, 2.0, 6.0, 80.0, 4.0, 80.0, kap) -
             concentric_cavity_solvation(1.0, 4.0, 2.0, 6.0, 4.0, 4.0, 80.0, kap))
    # the cavity's effect (about 7 % of the energy) to the meshes' error: 6.4 %
    # with a 320-panel cavity, 2.1 % with 1280 panels
    assert (out[80.0] - out[4.0]) == pytest.approx(d_ref, rel=0.04)


def test_interface_between_equal_media_changes_nothing():
    """A shell whose interior is the solvent itself (same eps and kappa)
    around a charged sphere: the energies equal those without the shell, to
    the discretisation error of the extra surface."""
    kap = 0.125
    m, s = _mol(2, 4.0, at=(0.5, 0.3, 0.0)), _shell(2, 6.0, 80.0)
    e_shell = _energy([m, s], kap, parent=[1, -1], kappa_in=[0.0, kap])
    e_plain = _energy([m], kap)
    assert e_shell["solvation"] == pytest.approx(e_plain["solvation"], rel=3e-3)


def test_series_limits():
    """The cavity series: the cavity's permittivity equal to the molecule's
    and the charge at the centre give the screened Born energy, which is the
    Stern closed form with b = a."""
    born = stern_sphere_solvation(1.0, 4.0, 4.0, 4.0, 80.0, 0.125)
    # (the off-centre terms are of relative size (c/b)^2 = 6e-8)
    assert concentric_cavity_solvation(1.0, 1e-3, 1e-4, 4.0, 4.0, 4.0, 80.0, 0.125, lmax=10) == \
        pytest.approx(born, rel=1e-6)
    # kappa = 0: Born's formula
    born0 = 0.5 * (1.0 / 80.0 - 1.0 / 4.0) / 4.0 * units.COULOMB_KCAL
    assert stern_sphere_solvation(1.0, 4.0, 6.0, 4.0, 80.0, 0.0) == pytest.approx(born0, rel=1e-12)


def _stern_bodies():
    v1, f1 = synth.icosphere(1, 4.0)
    v2, f2 = synth.icosphere(1, 6.0)
    return [Body(DIELECTRIC, v1, f1, eps_in=4.0, charge_xyz=np.array([[0.5, 0.0, 0.0]]), charge_q=np.array([1.0])),
            Body(DIELECTRIC, v2, f2, eps_in=80.0)]


def test_region_treecode_at_theta_zero_is_the_dense_rows():
    """theta = 0: every node is opened, so the per-region treecode is the
    direct sum of the dense rows (to rounding)."""
    from oracle.regions import RegionTreecode
    rs = RegionSystem(_stern_bodies(), 80.0, 0.125, parent=[1, -1], params=Params(theta=0.0, leaf_size=8))
    x = np.random.default_rng(1).normal(size=rs.n)
    ref = rs.assemble()[0] @ x
    y = RegionTreecode(rs).apply(x)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_region_treecode_converges_with_P():
    from oracle.regions import RegionTreecode
    bodies = _stern_bodies()
    A = RegionSystem(bodies, 80.0, 0.125, parent=[1, -1]).assemble()[0]
    x = np.random.default_rng(1).normal(size=A.shape[0])
    ref = A @ x
    errs = []
    for P in (2, 4, 6):
        rs = RegionSystem(bodies, 80.0, 0.125, parent=[1, -1], params=Params(theta=0.5, P=P, leaf_size=8))
        errs.append(np.abs(RegionTreecode(rs).apply(x) - ref).max() / np.abs(ref).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-4


def test_region_treecode_without_nesting_is_the_plain_treecode():
    """No nesting: the per-region passes (molecule interior, solvent) give
    exactly the fused treecode of oracle.treecode."""
    from oracle.regions import RegionTreecode
    from oracle.treecode import TreecodeOperator
    v1, f1 = synth.icosphere(1, 4.0)
    v2, f2 = synth.icosphere(0, 3.0)
    bodies = [Body(DIELECTRIC, v1, f1, eps_in=4.0, charge_xyz=np.array([[0.3, 0.0, 0.0]]), charge_q=np.array([1.0])),
              Body(SET_CHARGE, v2 + [9.0, 0, 0], f2, bc_value=units.sigma_from_c_m2(0.05))]
    prm = Params(theta=0.5, P=4, leaf_size=8)
    x = np.random.default_rng(2).normal(size=RegionSystem(bodies, 80.0, 0.125).n)
    ya = RegionTreecode(RegionSystem(bodies, 80.0, 0.125, params=prm)).apply(x)
    yb = TreecodeOperator(System(bodies, 80.0, 0.125, prm)).apply(x)
    assert np.abs(ya - yb).max() <= 1e-13 * np.abs(yb).max()


def test_charged_surface_behind_an_interface_between_equal_media():
    """An imposed-charge sphere and a molecule, both inside a shell whose
    interior is the solvent itself (same eps and kappa): surface and
    solvation energies equal those without the shell, so the rows of a
    surface in a region other than the solvent (its imposed density
    -sigma0 / eps_R) and the surface energy there are consistent."""
    kap = 0.125
    vm, fm = synth.icosphere(2, 3.0)
    vs, fs = synth.icosphere(1, 2.0)
    vb, fb = synth.icosphere(2, 12.0)
    mol = Body(DIELECTRIC, vm + [-4.0, 0, 0], fm, eps_in=4.0, charge_xyz=np.array([[-4.0, 0.2, 0.0]]),
               charge_q=np.array([1.0]))
    srf = Body(SET_CHARGE, vs + [4.0, 0, 0], fs, bc_value=units.sigma_from_c_m2(0.05))
    shell = Body(DIELECTRIC, vb, fb, eps_in=80.0)
    e_in = _energy([mol, srf, shell], kap, parent=[2, 2, -1], kappa_in=[0.0, 0.0, kap])
    e_plain = _energy([mol, srf], kap)
    for k in ("solvation", "surface", "total"):
        assert e_in[k] == pytest.approx(e_plain[k], rel=2e-3)
    # and the test sees the medium: an unscreened interior moves the surface energy by 30 %
    e_bad = _energy([mol, srf, shell], kap, parent=[2, 2, -1], kappa_in=[0.0, 0.0, 0.0])
    assert abs(e_bad["surface"] - e_plain["surface"]) > 0.1 * abs(e_plain["surface"])
