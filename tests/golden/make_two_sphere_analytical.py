"""Writes two_sphere_analytical.txt: the analytical two-sphere energies
(Section 4: Eq. 17 interaction energy from the series solution, Eq. 32-44)
for the paper's grid-convergence geometry (Section 5.1: a dielectric sphere of
radius 5 A with a central unit charge, eps 4, and a sphere of radius 4 A held
at potential phi0 = 1 internal unit, centres 12 A apart, kappa 0.125 1/A,
eps 80) and for the same pair with both radii 4 A, charged (0.05 C/m^2) and
held at 0.05 V.  The series is taken to N = 40 and to N = 60; the file
records both (they agree to round-off).  Calls only oracle/; run from the
repository root:
    python tests/golden/make_two_sphere_analytical.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path[:0] = [ROOT]

from oracle import units  # noqa: E402
from oracle.analytical import interaction  # noqa: E402

CASES = {
    # name: (d1, d2, R, q, eps1, eps2, kappa, phi0 (internal), sigma0 (internal))
    "paper_5_4_phi1": (5.0, 4.0, 12.0, 1.0, 4.0, 80.0, 0.125, 1.0, None),
    "pair_4_4_sigma005": (4.0, 4.0, 12.0, 1.0, 4.0, 80.0, 0.125, None, units.sigma_from_c_m2(0.05)),
    "pair_4_4_phi005": (4.0, 4.0, 12.0, 1.0, 4.0, 80.0, 0.125, units.phi_from_volt(0.05), None),
}


def main():
    out = os.path.join(HERE, "two_sphere_analytical.txt")
    with open(out, "w") as fh:
        fh.write("# analytical two-sphere energies (kcal/mol): case N F_int solv surf iso_mol iso_surf\n")
        fh.write(f"# one internal potential unit = {units.POTENTIAL_VOLT:.17e} V\n")
        for name, (d1, d2, R, q, e1, e2, k, phi0, sig0) in CASES.items():
            for N in (40, 60):
                F, parts = interaction(d1, d2, R, q, e1, e2, k, phi0=phi0, sigma0=sig0, N=N)
                fh.write(f"{name} {N} {F:.17e} {parts['solv']:.17e} {parts['surf']:.17e} "
                         f"{parts['iso_mol']:.17e} {parts['iso_surf']:.17e}\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
