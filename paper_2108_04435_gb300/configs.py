"""Workload presets shaped like the paper's runs, in lattice units.

Temperature presets (alpha, alpha' at 1.6 K and 1.9 K) are the values the
workload definitions quote; rho_s/rho_n, kappa in lattice units and the core
radius are readings (the paper prints none of them): kappa_LB follows from
matching the lattice viscosity (tau - 1/2)/3 to nu_n(T) at tau = 0.6, and the
core radius a ~ 1 Angstrom (Sec. I) is expressed in cells of 2 mm / 64.
"""
from __future__ import annotations

import numpy as np

from . import inputs

DX_CM = 0.2 / 64.0          # Sec. III: L_x = 2 mm over 64 cells
CORE_A = 1.3e-8 / DX_CM     # core radius ~ 1 Angstrom in cells

TEMPS = {
    # T: alpha, alpha', rho_s/rho_n, kappa in lattice units (tau = 0.6)
    1.9: dict(alpha=0.206, alpha_p=0.0083, rho_s_over_rho_n=1.38, kappa=0.157),
    1.6: dict(alpha=0.098, alpha_p=0.016, rho_s_over_rho_n=5.2, kappa=0.057),
    # 2.1 K: approximate values (not given by the paper or the workload definitions)
    2.1: dict(alpha=0.5, alpha_p=0.02, rho_s_over_rho_n=0.35, kappa=0.22),
}


def base_params(n, wall, T=1.9, **kw):
    p = dict(n=list(n), wall=list(wall), stream_axis=2, vfm_substeps=1, couple=1, force_form=0,
             max_points=4096, storage=0, wall_images=0, tau=0.6, rho0=1.0, body_force=[0.0, 0.0, 0.0],
             heater_vn=0.0, pin_vn=0.0, init_vn=[0.0, 0.0, 0.0], core_a=CORE_A,
             dxi_min=0.70, dxi_max=0.95)
    p.update(TEMPS[T])
    p.update(kw)
    return p


def counterflow_vn(v_ns: float, T: float) -> float:
    """Normal velocity giving counterflow v_ns with V_s from Eq. 18 (box mean)."""
    r = TEMPS[T]["rho_s_over_rho_n"]
    return v_ns * r / (1.0 + r)


def config(name: str, seed: int = 0):
    """Return (params, xyz, next) for one of the named workloads."""
    if name == "ring32":
        # 32^3 periodic, one ring R = 8 (64 points), counterflow v_ns = 0.02 along z, 1.9 K
        p = base_params((32, 32, 32), (0, 0, 0), 1.9, max_points=512,
                        init_vn=[0.0, 0.0, counterflow_vn(0.02, 1.9)])
        xyz, nxt = inputs.ring((16.0, 16.0, 16.0), (0.0, 0.0, 1.0), 8.0, npts=64)
        return p, xyz, nxt
    if name == "channel64x64x256":
        # closed channel, walls on all sides, heater v_n = 0.01 along z, 20 rings R ~ U[4, 12]
        p = base_params((64, 64, 256), (1, 1, 1), 1.9, heater_vn=0.01, init_vn=[0.0, 0.0, 0.01],
                        max_points=8192)
        xyz, nxt = inputs.random_rings((64, 64, 256), (1, 1, 1), 20, 4.0, 12.0, seed)
        return p, xyz, nxt
    if name == "box128":
        # 128^3 periodic counterflow v_ns = 0.03, 200 rings R ~ U[6, 20]
        p = base_params((128, 128, 128), (0, 0, 0), 1.9, max_points=65536,
                        init_vn=[0.0, 0.0, counterflow_vn(0.03, 1.9)])
        xyz, nxt = inputs.random_rings((128, 128, 128), (0, 0, 0), 200, 6.0, 20.0, seed)
        return p, xyz, nxt
    if name == "channel128x128x1024":
        # closed channel ~16.8M cells, 1.6 K, 1000 rings R ~ U[6, 20]
        p = base_params((128, 128, 1024), (1, 1, 1), 1.6, heater_vn=0.01, init_vn=[0.0, 0.0, 0.01],
                        max_points=262144)
        xyz, nxt = inputs.random_rings((128, 128, 1024), (1, 1, 1), 1000, 6.0, 20.0, seed)
        return p, xyz, nxt
    if name == "channel64x64x256_lines":
        # the closed channel of Sec. IV seeded as there: four lines bound to the heater and the far
        # wall, with a helical kink, and two smaller rings to kick them; heater v_n = 0.01 along z
        p = base_params((64, 64, 256), (1, 1, 1), 1.9, heater_vn=0.01, init_vn=[0.0, 0.0, 0.01],
                        max_points=8192)
        lines = inputs.wall_lines((64, 64, 256), 4, seed, amp=2.0)
        for k in range(1, 64):  # rings redrawn until they pass 3 cells clear of the lines
            rings = inputs.random_rings((64, 64, 256), (1, 1, 1), 2, 5.0, 7.0, seed + k)
            gap = np.sqrt(((rings[0][:, None, :] - lines[0][None, :, :]) ** 2).sum(-1)).min()
            if gap >= 3.0:
                break
        xyz, nxt = inputs.concat([lines, rings])
        return p, xyz, nxt
    raise KeyError(name)


NAMES = ["ring32", "channel64x64x256", "box128", "channel128x128x1024", "channel64x64x256_lines"]


MACH_SAFE_VN = 0.02  # imposed |u| with headroom under the Mach limit 0.05 c_s = 0.0289 (Sec. II.B)


def serving_requests(count: int, rate: float, seed: int, steps: int,
                     grids=((32, 32, 32), (64, 64, 64), (64, 64, 256), (128, 128, 128)),
                     temps=(1.6, 1.9, 2.1), vns=(0.005, 0.04), points=(100, 20000), storage: int = 0):
    """Seeded counterflow requests arriving as a Poisson process of `rate`/s.

    Each request: a periodic grid from `grids`, a temperature from `temps`,
    a counterflow v_ns ~ U[vns] (the normal velocity it implies is capped at
    MACH_SAFE_VN), and rings seeded until about U[points] filament points,
    capped at a line density of 0.02 per cell^2 of the grid.
    Returns a list of dicts with arrival time, params, xyz, next and steps.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    for k in range(count):
        t += rng.exponential(1.0 / rate)
        n = grids[int(rng.integers(len(grids)))]
        T = temps[int(rng.integers(len(temps)))]
        v_ns = rng.uniform(*vns)
        target = int(rng.uniform(*points))
        target = min(target, int(0.02 * n[0] * n[1] * n[2] / 0.8))
        r_max = min(n) / 4.0 - 3.0
        r_min = min(4.0, r_max)
        mean_pts = 2 * np.pi * 0.5 * (r_min + r_max) / 0.8
        count_rings = max(1, int(round(target / mean_pts)))
        xyz, nxt = inputs.random_rings(n, (0, 0, 0), count_rings, r_min, r_max, seed * 100003 + k, min_sep=2.0,
                                       max_tries=20, skip_crowded=True)
        vn = min(counterflow_vn(v_ns, T), MACH_SAFE_VN)
        p = base_params(n, (0, 0, 0), T, init_vn=[0.0, 0.0, vn], storage=storage,
                        max_points=max(4096, int(4 * len(nxt))))
        out.append(dict(id=k, arrival=t, params=p, xyz=xyz, next=nxt, steps=steps, grid=n, T=T, v_ns=v_ns))
    return out
