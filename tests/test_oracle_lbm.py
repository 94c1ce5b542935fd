"""Pins of the oracle's lattice-Boltzmann pass (Sec. II.B, Eqs. 5-9, 12-14, 18).

Closed forms: uniform flow is a fixed point; body-force Poiseuille flow with
halfway bounce-back at the BGK "magic" relaxation time tau = 1/2 + sqrt(3)/4
is exact (this pins the half-force velocity shift and the wall rule); the
Taylor-Green mode decays at exp(-2 nu k^2 t); mass is conserved with periodic
axes, walls and the heater; the heater channel relaxes to plug counterflow
with V_s = -(rho_n/rho_s) v_n (Eq. 18), i.e. v_ns = v_n rho/rho_s (Eqs. 1-2).
"""
import numpy as np
import pytest

from paper_2108_04435_gb300 import configs, inputs


def params(n, wall, **kw):
    kw.setdefault("couple", 0)
    kw.setdefault("max_points", 8)
    return configs.base_params(n, wall, 1.9, **kw)


def test_uniform_flow_is_fixed_point(oracle_mod):
    p = params((6, 5, 7), (0, 0, 0), init_vn=[0.01, -0.02, 0.015])
    ch = oracle_mod.Channel(p)
    f0 = ch.read(oracle_mod.FIELD_FSTAR)
    ch.step(10)
    f1 = ch.read(oracle_mod.FIELD_FSTAR)
    assert np.abs(f1 - f0).max() < 2e-15


def test_heater_uniform_plug_flow_is_fixed_point(oracle_mod):
    """f^eq(rho0, v e_z) satisfies the moving-wall links at both heater faces."""
    p = params((3, 4, 9), (0, 0, 1), heater_vn=0.01, init_vn=[0.0, 0.0, 0.01])
    ch = oracle_mod.Channel(p)
    f0 = ch.read(oracle_mod.FIELD_FSTAR)
    ch.step(10)
    assert np.abs(ch.read(oracle_mod.FIELD_FSTAR) - f0).max() < 2e-15
    vs = ch.read(oracle_mod.FIELD_PLANE_VS)
    assert np.abs(vs - (-0.01 / p["rho_s_over_rho_n"])).max() < 1e-15


@pytest.mark.parametrize("wall,heater", [((0, 0, 0), 0.0), ((1, 1, 1), 0.0), ((1, 0, 1), 0.01)])
def test_mass_conservation(oracle_mod, wall, heater):
    n = (6, 5, 8)
    p = params(n, wall, heater_vn=heater, init_vn=[0.0, 0.0, heater])
    ch = oracle_mod.Channel(p)
    ncell = n[0] * n[1] * n[2]
    f0 = ch.read(oracle_mod.FIELD_FSTAR) * inputs.perturbed_equilibrium(ncell, 3, 1e-2)
    ch.write(oracle_mod.FIELD_FSTAR, f0)
    F = inputs.random_field((3, ncell), 4, 1e-4)
    ch.write(oracle_mod.FIELD_FORCE, F)
    ch.step(1)
    m0 = ch.stats()[2]
    ch.step(200)
    m1 = ch.stats()[2]
    assert abs(m1 / m0 - 1.0) < 1e-13


def test_poiseuille_magic_tau_exact(oracle_mod):
    H, g = 16, 1e-5
    tau = 0.5 + np.sqrt(3.0) / 4.0
    p = params((1, H, 1), (0, 1, 0), tau=tau, body_force=[g, 0.0, 0.0])
    ch = oracle_mod.Channel(p)
    ch.step(6000)
    u = ch.read(oracle_mod.FIELD_U)[0]
    nu = (tau - 0.5) / 3.0
    y = np.arange(H)
    exact = g / (2 * nu) * ((H / 2.0) ** 2 - (y - (H - 1) / 2.0) ** 2)
    assert np.abs(u / exact - 1.0).max() < 1e-9


def test_poiseuille_without_shift_would_fail(oracle_mod):
    """The exact profile needs u = (sum c f + F/2)/rho; the unshifted moment is
    off by F/(2 rho), far outside the tolerance above."""
    H, g = 16, 1e-5
    tau = 0.5 + np.sqrt(3.0) / 4.0
    p = params((1, H, 1), (0, 1, 0), tau=tau, body_force=[g, 0.0, 0.0])
    ch = oracle_mod.Channel(p)
    ch.step(6000)
    u = ch.read(oracle_mod.FIELD_U)[0]
    unshifted = u - 0.5 * g / ch.read(oracle_mod.FIELD_RHO)
    nu = (tau - 0.5) / 3.0
    y = np.arange(H)
    exact = g / (2 * nu) * ((H / 2.0) ** 2 - (y - (H - 1) / 2.0) ** 2)
    assert np.abs(unshifted / exact - 1.0).max() > 1e-4


def test_taylor_green_decay(oracle_mod):
    n = 32
    p = params((n, n, 1), (0, 0, 0))
    ch = oracle_mod.Channel(p)
    x, y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    k = 2 * np.pi / n
    U0 = 0.01
    ux = U0 * np.sin(k * x) * np.cos(k * y)
    uy = -U0 * np.cos(k * x) * np.sin(k * y)
    rho = 1.0 - 3.0 * U0 ** 2 / 4.0 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    f = np.stack([oracle_mod.feq(r, [a, b, 0.0]) for r, a, b in zip(rho.ravel(), ux.ravel(), uy.ravel())], axis=1)
    ch.write(oracle_mod.FIELD_FSTAR, f)
    e0 = (ch.read(oracle_mod.FIELD_U) ** 2).sum()
    ch.step(200)
    e1 = (ch.read(oracle_mod.FIELD_U) ** 2).sum()
    nu = (p["tau"] - 0.5) / 3.0
    rate = np.log(e1 / e0) / 200
    assert abs(rate / (-2 * nu * 2 * k * k) - 1.0) < 0.01


def test_heater_counterflow_relation(oracle_mod):
    """Closed channel (walls on the stream axis) started at rest relaxes to
    plug flow v_n = heater_vn, so Eq. 18 gives V_s = -(rho_n/rho_s) v_n and
    v_ns = v_n - V_s = v_n rho/rho_s, which is Eq. 2 with v_n = W/(A rho sigma T)."""
    v = 0.01
    p = params((4, 4, 16), (0, 0, 1), tau=1.0, heater_vn=v)
    ch = oracle_mod.Channel(p)
    ch.step(3000)
    vs = ch.read(oracle_mod.FIELD_PLANE_VS)
    r = p["rho_s_over_rho_n"]
    assert np.abs(vs / (-v / r) - 1.0).max() < 1e-6
    vns = v - vs
    assert np.abs(vns / (v * (1.0 + r) / r) - 1.0).max() < 1e-6
    assert abs(ch.stats()[2] / (4 * 4 * 16) - 1.0) < 1e-12


def test_mach_limit_reported(oracle_mod):
    """Sec. II.B requires |u|/c_s < 0.05; a faster flow is an error."""
    p = params((4, 4, 4), (0, 0, 0), init_vn=[0.04, 0.0, 0.0])
    ch = oracle_mod.Channel(p)
    rc = ch.step(1, check=False)
    assert rc == -5
    assert abs(ch.stats()[4] - 0.04 * np.sqrt(3.0)) < 1e-12
