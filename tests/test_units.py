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


def test_line_density_fit_recovers_a_linear_profile():
    # Sec. IV: L(z) = L0 (1 - z/z0) through the plane centres of the 64-cell
    # channel (2 mm), with zero-mean noise that a least-squares line ignores
    z = [(k + 0.5) * 2.0 / 64 for k in range(64)]
    L0, z0 = 1500.0, 3.2
    prof = [L0 * (1 - zk / z0) + (5.0 if k % 2 else -5.0) for k, zk in enumerate(z)]
    fL0, fz0 = tangle.line_density_fit(z, prof)
    assert fL0 == pytest.approx(L0, rel=1e-2)
    assert fz0 == pytest.approx(z0, rel=2e-2)
    exact = tangle.line_density_fit(z, [L0 * (1 - zk / z0) for zk in z])
    assert exact == pytest.approx((L0, z0), rel=1e-12)
    # a flat profile: z0 (where the fit reaches zero) lies far beyond the channel
    fL0, fz0 = tangle.line_density_fit(z, [L0] * 64)
    assert fL0 == pytest.approx(L0, rel=1e-12) and abs(fz0) > 1e9


def test_delta_T_in_SI_units():
    # delta T = (alpha / sigma) kappa L0 V_ns (Eq. 20), evaluated here in SI:
    # kappa 9.97e-8 m^2/s, L0 1000 cm^-2 = 1e7 m^-2, V_ns 0.5 cm/s = 5e-3 m/s,
    # sigma 0.757e7 erg/(g K) = 757 J/(kg K); K/m -> mK/m
    alpha = 0.098
    si = alpha / 757.0 * 9.97e-8 * 1e7 * 5e-3 * 1e3
    assert tangle.delta_T_mK_per_m(alpha, 1000.0, 0.5) == pytest.approx(si, rel=1e-12)


def test_temperature_profile_solves_the_gradient_relation():
    # Eq. 20 must integrate Eq. 19, dT/dz = -(alpha/sigma) kappa L(z) V_ns,
    # for L(z) = L0 (1 - z/z0): integrate the right side numerically (the
    # trapezoid rule is exact for a linear integrand) and compare
    dT, z0, T0 = 2.0e-3, 3.2, 1.9
    z = [k * 2.0 / 400 for k in range(401)]
    grad = [-dT * (1 - zk / z0) for zk in z]  # -(alpha/sigma) kappa V_ns L(z) = -dT L(z)/L0
    T = [T0]
    for k in range(1, len(z)):
        T.append(T[-1] + 0.5 * (grad[k] + grad[k - 1]) * (z[k] - z[k - 1]))
    assert list(tangle.temperature_profile(z, T0, dT, z0)) == pytest.approx(T, rel=0, abs=1e-15)
    # the drop across the channel is below dT * length for z0 beyond the channel
    assert tangle.temperature_profile([2.0], T0, dT, z0)[0] > T0 - dT * 2.0
