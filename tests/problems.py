"""Shared seeded test problems: the same synthetic bodies handed to the CUDA
library (through the C ABI) and to the CPU oracle."""
import numpy as np

import synth
from oracle import units
from oracle.bem import DIELECTRIC, SET_CHARGE, SET_POTENTIAL, Body, Params, System

KIND = {"dielectric": DIELECTRIC, "sigma": SET_CHARGE, "phi": SET_POTENTIAL}


def spheres(level_mol=2, level_srf=2, r_mol=4.0, r_srf=4.0, sep=12.0, kind="sigma", bc=0.05, surface=True,
            mol_nu=None):
    """Molecule sphere (central +1e) and an imposed-charge/potential sphere
    `sep` apart along x.  bc in C/m^2 (sigma) or V (phi).  mol_nu: use a
    geodesic frequency-nu sphere for the molecule instead (ragged sizes)."""
    if mol_nu:
        v, f = synth.geodesic_sphere(mol_nu)
        v = v * r_mol
    else:
        v, f = synth.icosphere(level_mol, r_mol)
    bodies = [dict(kind="dielectric", verts=v, tris=f, eps_in=4.0, qxyz=np.zeros((1, 3)), q=np.array([1.0]), bc=0.0)]
    if surface:
        v2, f2 = synth.icosphere(level_srf, r_srf)
        bodies.append(dict(kind=kind, verts=v2 + np.array([sep, 0.0, 0.0]), tris=f2, eps_in=1.0,
                           qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=bc))
    return bodies


def star_molecule(seed=3, nu=10, nq=60, r0=15.0):
    v, f = synth.star_surface(seed, nu, r0)
    coeffs = synth.star_coefficients(seed)
    xyz, q = synth.interior_charges(seed, nq, v, f, radius_fn=lambda d: synth.star_radius(d, coeffs, r0))
    return [dict(kind="dielectric", verts=v, tris=f, eps_in=4.0, qxyz=xyz, q=q, bc=0.0)]


def oracle_system(bodies, eps_out=80.0, kappa=0.125, **params):
    ob = []
    for b in bodies:
        k = KIND[b["kind"]]
        bc = units.sigma_from_c_m2(b["bc"]) if k == SET_CHARGE else (units.phi_from_volt(b["bc"]) if k == SET_POTENTIAL else 0.0)
        ob.append(Body(k, b["verts"], b["tris"], eps_in=b["eps_in"], charge_xyz=b["qxyz"], charge_q=b["q"],
                       bc_value=bc, R=b.get("R"), t=b.get("t")))
    return System(ob, eps_out, kappa, Params(**params))


def gpu_context(bodies, eps_out=80.0, kappa=0.125, **params):
    from paper_1506_03745_gb300.context import context
    return context(bodies, eps_out, kappa, **params)
