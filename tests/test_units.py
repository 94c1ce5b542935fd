"""Unit conversion of the physical-unit runs (Sec. III.C, Sec. IV).

The lattice units must keep the dimensionless groups of the physical run:
kappa / nu_n (the ratio that sets the coupling), V_n dt / dx (the lattice
velocity, here 0.02 at 2.5 mm/s) and the paper's dx = 2 mm / 64 (Sec. III),
which also makes the Sec. III.A ring of 0.24 mm 7.68 cells
(tests/golden/paper_units.txt)."""
import math

import pytest

from paper_2108_04435_gb300 import configs, tangle


def test_dimensionless_groups():
    u = tangle.units(2.5, u_max=0.02)
    assert u["dx_cm"] == pytest.approx(0.2 / 64, rel=1e-15)
    # kappa_LB / nu_LB = kappa / nu_n
    assert u["kappa_lb"] / u["nu_lb"] == pytest.approx(tangle.HE_19K["kappa_over_nu_n"], rel=1e-12)
    # tau from the lattice viscosity nu = (tau - 1/2) / 3
    assert (u["tau"] - 0.5) / 3.0 == pytest.approx(u["nu_lb"], rel=1e-12)
    # 2.5 mm/s is 0.02 cells per step, under the Mach limit |u| sqrt(3) < 0.05
    p = tangle.t1_params(2.5, u)
    assert p["pin_vn"] == pytest.approx(0.02, rel=1e-12)
    assert math.sqrt(3.0) * p["pin_vn"] < 0.05
    assert tangle.t1_params(2.0, u)["pin_vn"] == pytest.approx(0.016, rel=1e-12)
    # rho_s / rho_n from rho_s / rho
    r = tangle.HE_19K["rho_s_over_rho"]
    assert u["rho_s_over_rho_n"] == pytest.approx(r / (1 - r), rel=1e-15)


def test_paper_ring_in_cells():
    assert 0.024 / configs.DX_CM == pytest.approx(7.68, rel=1e-12)


def test_line_density_conversion():
    u = tangle.units()
    n = tangle.BOX[0] * tangle.BOX[1] * tangle.BOX[2]
    # one cell of line per cell of volume is 1 / dx^2
    assert tangle.line_density_cm2(n, u) == pytest.approx(1.0 / u["dx_cm"] ** 2, rel=1e-15)
