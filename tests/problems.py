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


def gap_offset(verts, radius, gap):
    """x offset D such that the molecule (verts) translated by (D, 0, 0) has
    its closest vertex `gap` from the sphere of `radius` at the origin
    (bisection on the closest-vertex distance)."""
    v = np.asarray(verts)
    lo, hi = radius + gap - v[:, 0].min() - 50.0, radius + gap - v[:, 0].min() + 50.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        d = np.sqrt(((v + np.array([mid, 0.0, 0.0])) ** 2).sum(1)).min() - radius
        lo, hi = (mid, hi) if d < gap else (lo, mid)
    return 0.5 * (lo + hi)


def config4_coarse():
    """The differentiation workload's dense-oracle version: the star molecule
    (seed 3, r0 15 A, geodesic frequency 10: 2000 panels, 900 charges) 10 A
    from a sphere of radius 40 A (frequency 13: 3380 panels) holding
    sigma0 = -0.05 C/m^2; the molecule is posed at (D, 0, 0)."""
    v, f = synth.star_surface(3, 10, 15.0)
    coeffs = synth.star_coefficients(3)
    xyz, q = synth.interior_charges(3, 900, v, f, radius_fn=lambda d: synth.star_radius(d, coeffs, 15.0))
    u, fs = synth.geodesic_sphere(13)
    mol = dict(kind="dielectric", verts=v, tris=f, eps_in=4.0, qxyz=xyz, q=q, bc=0.0,
               R=np.eye(3), t=np.array([gap_offset(v, 40.0, 10.0), 0.0, 0.0]))
    srf = dict(kind="sigma", verts=u * 40.0, tris=fs, eps_in=1.0, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=-0.05,
               R=np.eye(3), t=np.zeros(3))
    return [mol, srf]


def fullsize_bodies():
    """The benchmark's two-sphere workload: molecule and imposed-charge
    (0.05 C/m^2) spheres of radius 4 A, icosphere level 5 (20480 panels
    each), centres 12 A apart, one +1e charge at the molecule's centre."""
    return spheres(level_mol=5, level_srf=5, kind="sigma", bc=0.05)


def fullsize_groups():
    """Eight target groups of the full-size workload (640 per body): the
    first, two inner and the last group of each body."""
    return [0, 211, 422, 639, 640, 851, 1062, 1279]


def fullsize_vectors(n):
    """Seeded density vectors: 'positive' (U(0.5, 1.5): every row a sum of
    terms of one sign up to the near-field corrections) and 'normal'."""
    return {"positive": np.random.default_rng(71).uniform(0.5, 1.5, size=n),
            "normal": np.random.default_rng(72).normal(size=n)}
