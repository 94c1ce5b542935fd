"""The counterflow tangle of Sec. III.C (T-1 regime) in physical units, and
the closed channel of Sec. IV.

The paper's box is 64 x 32 x 32 cells with L = 2 mm along the counterflow,
all faces periodic, at T = 1.9 K; the normal velocity V_n (2.0 - 2.5 mm/s)
is held by resetting the populations of the plane at the channel's ends to
equilibrium at V_n, and V_s follows from Eq. 18.  It reports a saturated line
density L_sat ~ 2000 cm^-2 at 2.0 mm/s and ~ 3500 cm^-2 at 2.5 mm/s, and
sqrt(L_sat) = gamma V_ns with gamma = 142 +- 17 s/cm^2.

Units.  The paper fixes dx = 2 mm / 64 but not dt (it mentions the sound
velocity and L_x only).  Here dt is chosen so that the largest V_n is 0.02
lattice units (Mach headroom under 0.05 c_s), and tau follows from matching
the lattice viscosity (tau - 1/2)/3 to nu_n dt/dx^2; kappa in lattice units is
kappa dt/dx^2.  The helium constants at 1.9 K (kappa/nu_n, rho_s/rho) are the
standard tabulated values, approximate and not printed by the paper.

The counterflow runs along z here (x in the paper): the lattice is
32 x 32 x 64.  Runs go through the public API (vlb.Channel) on the GPU.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import configs, inputs

KAPPA_CM2_S = 9.97e-4          # h / m_4
HE_19K = dict(T=1.9, kappa_over_nu_n=4.7, rho_s_over_rho=0.58)  # approximate He II values at 1.9 K
BOX = (32, 32, 64)             # cells; z = the counterflow axis (L_z = 2 mm)


def units(vn_max_mm_s: float = 2.5, u_max: float = 0.02, dx_cm: float = configs.DX_CM, he=HE_19K):
    """dt, tau and kappa in lattice units for the given velocity scale."""
    dt = u_max * dx_cm / (0.1 * vn_max_mm_s)           # V_n max -> u_max cells per step
    nu_n = KAPPA_CM2_S / he["kappa_over_nu_n"]          # cm^2/s
    nu_lb = nu_n * dt / dx_cm ** 2
    return dict(dx_cm=dx_cm, dt_s=dt, tau=0.5 + 3.0 * nu_lb, kappa_lb=KAPPA_CM2_S * dt / dx_cm ** 2,
                nu_lb=nu_lb, rho_s_over_rho_n=he["rho_s_over_rho"] / (1.0 - he["rho_s_over_rho"]))


def t1_params(vn_mm_s: float, u=None, max_points: int = 65536):
    """Channel parameters of the T-1 run at normal velocity vn_mm_s."""
    u = u or units()
    vn_lb = 0.1 * vn_mm_s * u["dt_s"] / u["dx_cm"]
    p = configs.base_params(BOX, (0, 0, 0), 1.9, tau=u["tau"], kappa=u["kappa_lb"],
                            rho_s_over_rho_n=u["rho_s_over_rho_n"], pin_vn=vn_lb,
                            init_vn=[0.0, 0.0, vn_lb], max_points=max_points)
    return p


def seed_rings(seed: int, count: int = 16):
    """Seed rings (the paper's seeds are not specified; the steady state
    should not depend on them, Sec. III.C)."""
    return inputs.random_rings(BOX, (0, 0, 0), count, 3.0, 7.0, seed)


def line_density_cm2(length_cells: float, u) -> float:
    """Line length per volume, L = length / V, in cm^-2."""
    ncell = BOX[0] * BOX[1] * BOX[2]
    return length_cells / (ncell * u["dx_cm"] ** 2)


def run(vn_mm_s: float, seconds: float, seed: int = 0, sample_s: float = 0.05, u=None):
    """One T-1 run on the GPU: L(t) in cm^-2, then L_sat over the last 40%
    of the run, V_ns = |V_n - V_s| in cm/s and gamma = sqrt(L_sat) / V_ns."""
    from . import vlb
    u = u or units()
    p = t1_params(vn_mm_s, u)
    xyz, nxt = seed_rings(seed)
    ch = vlb.Channel(p)
    ch.seed(xyz, nxt)
    steps = int(round(seconds / u["dt_s"]))
    every = max(1, int(round(sample_s / u["dt_s"])))
    t, L, vns = [], [], []
    t0 = time.perf_counter()
    done, error = 0, ""
    while done < steps:
        n = min(every, steps - done)
        try:
            ch.step(n)
        except vlb.VlbError as e:  # keep what was measured up to the failing step
            error = str(e)
            break
        done += n
        t.append(done * u["dt_s"])
        L.append(line_density_cm2(ch.line_length(), u))
        if done >= 0.6 * steps:
            uz = ch.read(vlb.FIELD_U)[2].mean()
            vs = ch.read(vlb.FIELD_PLANE_VS).mean()
            vns.append(abs(uz - vs) * u["dx_cm"] / u["dt_s"])
    wall = time.perf_counter() - t0
    st = ch.stats()
    ch.close()
    t, L = np.asarray(t), np.asarray(L)
    tail = t >= 0.6 * seconds
    L_sat = float(L[tail].mean()) if tail.any() else float("nan")
    V_ns = float(np.mean(vns)) if vns else float("nan")
    return dict(vn_mm_s=vn_mm_s, seconds=seconds, steps=done, error=error, seed=seed, dt_s=u["dt_s"], tau=u["tau"],
                kappa_lb=u["kappa_lb"], L_sat_cm2=L_sat, L_sat_std=float(L[tail].std()), V_ns_cm_s=V_ns,
                gamma=math.sqrt(L_sat) / V_ns if V_ns > 0 and L_sat > 0 else None, points=int(st[0]), status=int(st[1]),
                reconnections=int(st[7]), gpu_wall_s=wall, t=t.tolist(), L=L.tolist())


SIGMA_19K = 0.757e7  # entropy of He II at 1.9 K in erg/(g K), approximate tabulated value (not printed by the paper)


def line_density_fit(z_mm, prof):
    """Least-squares line through the averaged density profile, written as
    L(z) = L0 (1 - z/z0) (Sec. IV): L0 in the profile's unit, z0 in z's."""
    B, A = np.polyfit(np.asarray(z_mm, dtype=float), np.asarray(prof, dtype=float), 1)
    return float(A), float(-A / B) if B != 0 else float("inf")


def delta_T_mK_per_m(alpha: float, L0_cm2: float, V_ns_cm_s: float, sigma=SIGMA_19K) -> float:
    """delta T = (alpha / sigma) kappa L0 V_ns, the gradient scale of Eq. 20
    (the solution of Eq. 19 for L(z) = L0 (1 - z/z0)), from CGS inputs
    (L0 in cm^-2, V_ns in cm/s, sigma in erg/(g K)) to mK/m."""
    K_per_cm = alpha / sigma * KAPPA_CM2_S * L0_cm2 * V_ns_cm_s
    return K_per_cm * 1e3 * 1e2  # K -> mK, 1/cm -> 1/m


def temperature_profile(z, T0: float, dT: float, z0: float):
    """Eq. 20: T(z) = T0 - dT (1 - z/(2 z0)) z, the temperature along the
    channel for a linear line density, z measured from the heater wall."""
    z = np.asarray(z, dtype=float)
    return T0 - dT * (1.0 - z / (2.0 * z0)) * z


def channel_params(vn_mm_s: float = 2.5, u=None, wall_images: int = 1, max_points: int = 65536, tau=None):
    """The closed channel of Sec. IV: the box of Sec. III.C with solid walls at
    the two ends of the counterflow axis (heater at z = 0, cooled wall at the
    far end) and periodic side faces; V_n injected by the heater.  tau, when
    given, replaces the viscosity-matched value (a more viscous normal fluid)."""
    u = u or units()
    vn_lb = 0.1 * vn_mm_s * u["dt_s"] / u["dx_cm"]
    return configs.base_params(BOX, (0, 0, 1), 1.9, tau=tau if tau else u["tau"], kappa=u["kappa_lb"],
                               rho_s_over_rho_n=u["rho_s_over_rho_n"], heater_vn=vn_lb,
                               init_vn=[0.0, 0.0, vn_lb], wall_images=wall_images, max_points=max_points)


def channel_seeds(seed: int):
    """Four lines bound to the two end walls and two smaller rings to kick
    them (Sec. IV)."""
    lines = inputs.wall_lines(BOX, 4, seed, amp=0.0)
    for k in range(1, 64):  # rings redrawn until they pass 2.5 cells clear of the lines
        rings = inputs.random_rings(BOX, (0, 0, 1), 2, 3.0, 5.0, seed + k)
        gap = np.sqrt(((rings[0][:, None, :] - lines[0][None, :, :]) ** 2).sum(-1)).min()
        if gap >= 2.5:
            break
    return inputs.concat([lines, rings])


def channel_run(vn_mm_s: float = 2.5, seconds: float = 7.2, t_avg: float = 1.0, seed: int = 0,
                sample_s: float = 0.05, wall_images: int = 1, u=None, tau=None):
    """Sec. IV on the GPU: total line length L(t), the line density profile
    L(z) averaged over t >= t_avg, its linear fit L(z) = L0 (1 - z/z0), and the
    temperature gradient scale delta T of Eq. 20, (alpha / sigma) kappa L0 V_ns."""
    from . import vlb
    u = u or units()
    p = channel_params(vn_mm_s, u, wall_images, tau=tau)
    xyz, nxt = channel_seeds(seed)
    ch = vlb.Channel(p)
    ch.seed(xyz, nxt)
    steps = int(round(seconds / u["dt_s"]))
    every = max(1, int(round(sample_s / u["dt_s"])))
    nz = BOX[2]
    plane = BOX[0] * BOX[1] * u["dx_cm"] ** 2  # cm^2 of line per cell of length, per plane
    t, Ltot, prof, vns = [], [], np.zeros(nz), []
    nprof, done, error = 0, 0, ""
    t0 = time.perf_counter()
    while done < steps:
        n = min(every, steps - done)
        try:
            ch.step(n)
        except vlb.VlbError as e:
            error = str(e)
            break
        done += n
        t.append(done * u["dt_s"])
        Ltot.append(line_density_cm2(ch.line_length(), u))
        if t[-1] >= t_avg:
            prof += ch.read(vlb.FIELD_LINE_PROFILE) / plane
            nprof += 1
            uz = ch.read(vlb.FIELD_U)[2].mean()
            vs = ch.read(vlb.FIELD_PLANE_VS).mean()
            vns.append(abs(uz - vs) * u["dx_cm"] / u["dt_s"])
    wall = time.perf_counter() - t0
    st = ch.stats()
    ch.close()
    prof = prof / max(nprof, 1)
    z_mm = (np.arange(nz) + 0.5) * u["dx_cm"] * 10.0  # plane centres from the heater wall at -1/2
    V_ns = float(np.mean(vns)) if vns else float("nan")
    L0, z0 = line_density_fit(z_mm, prof)
    return dict(vn_mm_s=vn_mm_s, seconds=seconds, steps=done, error=error, wall_images=wall_images, tau=p["tau"],
                L_mean_cm2=float(np.mean(prof)), L0_cm2=L0, z0_mm=z0, V_ns_cm_s=V_ns,
                dT_mK_per_m=delta_T_mK_per_m(p["alpha"], L0, V_ns), points=int(st[0]), wall_cuts=int(st[13]),
                status=int(st[1]),
                gpu_wall_s=wall, t=t, L_total=Ltot, z_mm=z_mm.tolist(), L_profile=prof.tolist())


def main():
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--vn", type=float, nargs="+", default=[2.0, 2.25, 2.5], help="V_n in mm/s")
    ap.add_argument("--seconds", type=float, default=6.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None, help="write the runs (with L(t)) as JSON here")
    ap.add_argument("--channel", action="store_true", help="the closed channel of Sec. IV instead")
    ap.add_argument("--u-max", type=float, default=0.02, help="lattice velocity of 2.5 mm/s in the channel run")
    ap.add_argument("--tau", type=float, default=None,
                    help="channel run: BGK relaxation time instead of the viscosity-matched 0.516, which "
                         "goes unstable at the outflow wall once the tangle perturbs the flow")
    a = ap.parse_args()
    if a.channel:
        # the closed channel concentrates the flow around the dense tangle: more Mach headroom
        r = channel_run(seconds=a.seconds, seed=a.seed, u=units(2.5, u_max=a.u_max), tau=a.tau)
        print(json.dumps({k: v for k, v in r.items() if k not in ("t", "L_total", "z_mm", "L_profile")}))
        if a.out:
            with open(a.out, "w") as f:
                json.dump(r, f)
        return
    u = units(max(a.vn))
    runs = [run(v, a.seconds, a.seed, u=u) for v in a.vn]
    for r in runs:
        print(json.dumps({k: v for k, v in r.items() if k not in ("t", "L")}))
    if len(runs) >= 2:
        # sqrt(L_sat) = gamma V_ns: least-squares slope through the origin
        x = np.array([r["V_ns_cm_s"] for r in runs])
        y = np.sqrt([r["L_sat_cm2"] for r in runs])
        print(json.dumps({"gamma_fit": float((x * y).sum() / (x * x).sum())}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(dict(units=u, runs=runs), f)


if __name__ == "__main__":
    main()
