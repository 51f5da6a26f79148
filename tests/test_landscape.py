"""The orientation free-energy landscape (pgb_orientation_landscape, host
code of the library: Boltzmann weights over orientations at each gap)
against its closed forms."""
import math

import numpy as np

import paper_1506_03745_gb300 as pgb

KT = 0.0019872043 * 300.0


def test_equal_energies_give_uniform_weights():
    out = pgb.pgb_orientation_landscape(np.full(12, -5.0), 6, 2)
    for g in out:
        assert g["p_max"] == 1.0 / 6
        # -kT ln <e^{-F/kT}> of a constant is the constant
        assert math.isclose(g["free_energy_kcal_mol"], -5.0, rel_tol=1e-14)


def test_two_level_system():
    """Two orientations dF apart: p = 1 / (1 + e^{-dF/kT}) for the lower one and
    the average free energy F0 - kT ln((1 + e^{-dF/kT}) / 2)."""
    dF = 0.7
    F = np.array([[1.0, 3.0], [1.0 + dF, 3.0 + dF]]).reshape(-1)  # orientation-major, gap-minor
    out = pgb.pgb_orientation_landscape(F, 2, 2)
    for g, f0 in zip(out, (1.0, 3.0)):
        assert g["most_likely_orientation"] == 0
        assert math.isclose(g["p_max"], 1.0 / (1.0 + math.exp(-dF / KT)), rel_tol=1e-12)
        assert math.isclose(g["free_energy_kcal_mol"], f0 - KT * math.log((1.0 + math.exp(-dF / KT)) / 2.0),
                            rel_tol=1e-12)


def test_large_spread_does_not_overflow():
    F = np.array([-3000.0, -2900.0, 5000.0])
    out = pgb.pgb_orientation_landscape(F, 3, 1)
    assert out[0]["most_likely_orientation"] == 0 and out[0]["p_max"] == 1.0
    assert math.isclose(out[0]["free_energy_kcal_mol"], -3000.0 + KT * math.log(3.0), rel_tol=1e-12)


def test_argument_errors():
    import pytest
    with pytest.raises(pgb.PgbError):
        pgb.pgb_orientation_landscape(np.array([1.0, np.nan]), 2, 1)
    with pytest.raises(pgb.PgbError):
        pgb.pgb_orientation_landscape(np.array([1.0, 2.0]), 2, 1, temperature=0.0)
