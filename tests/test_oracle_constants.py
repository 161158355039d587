"""Pins of the oracle's unit constants (App. C) against the paper's printed
values and against scipy's CODATA table."""
import json
import math
import os

import pytest
from scipy import constants as sc

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_constants_match_paper_and_codata(orc):
    g = json.load(open(GOLD))
    c = orc.constants()
    # printed in App. C
    assert c["h"] == g["h_eV_ps"]
    assert c["mvv2e"] == g["mvv2e_eV_per_amu_A2_ps-2"]
    # independent: CODATA via scipy (h in eV s -> eV ps; amu A^2/ps^2 in eV)
    assert c["kB"] == pytest.approx(sc.k / sc.e, rel=1e-12)
    assert c["h"] == pytest.approx(sc.h / sc.e * 1e12, rel=1e-6)
    assert c["hbar"] == pytest.approx(c["h"] / (2 * math.pi), rel=1e-15)
    amu_A2_ps2_J = sc.physical_constants["atomic mass constant"][0] * 1e-20 / 1e-24
    assert c["mvv2e"] == pytest.approx(amu_A2_ps2_J / sc.e, rel=1e-6)


def test_de_boer_neon_worked_example(orc):
    """App. C: Lambda* for neon from the printed inputs.  Recomputed here in SI
    units from scipy's constants (independent of the oracle's metal-unit
    table); the printed 0.600 is off by 1.6% and is recorded, not asserted."""
    g = json.load(open(GOLD))["neon"]
    m_kg = g["m_g_per_mol"] * sc.physical_constants["atomic mass constant"][0]
    eps_J = g["eps_eV"] * sc.e
    sig_m = g["sigma_A"] * 1e-10
    lam_si = sc.h / (sig_m * math.sqrt(m_kg * eps_J))
    lam = orc.de_boer(g["m_g_per_mol"], g["eps_eV"], g["sigma_A"])
    assert lam == pytest.approx(lam_si, rel=2e-6)
    assert lam == pytest.approx(0.5906, abs=1e-4)
    printed = json.load(open(GOLD))["printed_lambda_star"]
    assert abs(printed - lam) / printed == pytest.approx(0.0158, abs=1e-3)
