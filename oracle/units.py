"""Unit system of the oracle (Section 2, Eq. 1).

Internal units: lengths in Angstrom, charge in e, relative permittivities, and
the vacuum permittivity set to one, so that Eq. 1 reads lap(phi) = -q delta/eps.
Potentials are then in e/(eps0*Angstrom), surface charge in e/Angstrom^2 and
energies in e^2/(eps0*Angstrom).  Conversions use CODATA 2018 exact/recommended
values.
"""
import math

E_CHARGE = 1.602176634e-19        # C (exact)
EPS0 = 8.8541878128e-12           # F/m
N_A = 6.02214076e23               # 1/mol (exact)
KCAL = 4184.0                     # J (thermochemical)
ANGSTROM = 1e-10                  # m

#: one internal energy unit e^2/(eps0*Angstrom) in kcal/mol (= 4*pi*332.0637...)
ENERGY_KCAL = E_CHARGE ** 2 / (EPS0 * ANGSTROM) * N_A / KCAL
#: Coulomb constant e^2/(4 pi eps0 Angstrom) in kcal/mol
COULOMB_KCAL = ENERGY_KCAL / (4.0 * math.pi)
#: one internal potential unit e/(eps0*Angstrom) in volts
POTENTIAL_VOLT = E_CHARGE / (EPS0 * ANGSTROM)


def sigma_from_c_m2(sigma_c_m2: float) -> float:
    """Surface charge density C/m^2 -> e/Angstrom^2."""
    return sigma_c_m2 / E_CHARGE * ANGSTROM ** 2


def phi_from_volt(phi_v: float) -> float:
    """Potential in volts -> internal potential unit e/(eps0*Angstrom)."""
    return phi_v / POTENTIAL_VOLT
