"""Further pins of the oracle: the pinned plane of Sec. III.C, the momentum
budget of one lattice pass (Eqs. 12-14), the magnitude of the mutual-friction
reaction of Eq. 10, and the direction of the merge priority of the remeshing.

- Pinned plane.  The periodic runs of Sec. III.C hold the normal velocity by
  setting it at the plane x = 0 = L_x.  The oracle resets that plane to the
  equilibrium of the cell's own pulled density and the imposed velocity.  A
  perturbed lattice makes the local density differ from rho0, so a reset with
  rho0, on another plane or with another velocity fails; a box at rest must
  relax to the uniform imposed flow.
- Momentum budget.  With Guo's split forcing, sum_i c_i f*_i = j + F for
  every cell (j the pulled momentum), and pull streaming on a periodic
  lattice moves populations without creating momentum: one pass adds exactly
  the summed force grid (and the body force on every cell) to the momentum.
- Friction reaction.  With the force read as the drag that balances the
  Magnus force (force_form 1), the normal fluid must receive the momentum the
  vortex loses: sum F = -(rho_s / rho_n) rho0 kappa dA/dt, where A is the
  vector area of the ring (its impulse is rho_s kappa A).  dA/dt is measured
  from the ring's own RK4 displacement over one step, independently of the
  force formula, so a wrong kappa, density ratio, rho0 or line-element
  weight fails.  (Form 0, Eq. 10 as printed, multiplies the same constant and
  line element; it is not momentum-conserving, so this balance cannot pin it.)
- Merge priority.  A point with short segments on both sides is removed
  unless a neighbouring candidate outranks it; rank is the MurmurHash3 32-bit
  finaliser of the point index, larger hash first.  The ring below has two
  candidate pairs and one candidate triple; the hashes are written out from
  the published finaliser, so reversing the comparison fails.
"""
import math

import numpy as np

from paper_2108_04435_gb300 import configs, inputs


def lparams(n, **kw):
    kw.setdefault("couple", 0)
    kw.setdefault("max_points", 8)
    return configs.base_params(n, (0, 0, 0), 1.9, **kw)


def pulled(oracle_mod, fstar, n):
    """Pull streaming on a periodic lattice: f_in,i(x) = f*_i(x - c_i)."""
    c, _, _ = oracle_mod.lattice()
    nx, ny, nz = n
    f = fstar.reshape(19, nz, ny, nx)
    out = np.empty_like(f)
    for i in range(19):
        out[i] = np.roll(f[i], shift=(c[i][2], c[i][1], c[i][0]), axis=(0, 1, 2))
    return out.reshape(19, -1)


def test_pinned_plane_resets_to_local_equilibrium(oracle_mod):
    n = (6, 5, 8)
    pin = 0.012
    p = lparams(n, pin_vn=pin)
    ch = oracle_mod.Channel(p)
    ncell = n[0] * n[1] * n[2]
    f0 = ch.read(oracle_mod.FIELD_FSTAR) * inputs.perturbed_equilibrium(ncell, 21, 2e-2)
    ch.write(oracle_mod.FIELD_FSTAR, f0)
    ch.run_phases(oracle_mod.PHASE_LBM)
    f1 = ch.read(oracle_mod.FIELD_FSTAR).reshape(19, n[2], n[1] * n[0])
    rho_local = pulled(oracle_mod, f0, n).sum(0).reshape(n[2], n[1] * n[0])
    assert np.abs(rho_local - 1.0).max() > 1e-3  # the local density is not rho0
    c, _, _ = oracle_mod.lattice()
    for k in range(n[1] * n[0]):
        want = oracle_mod.feq(rho_local[0, k], [0.0, 0.0, pin])
        assert np.abs(f1[:, 0, k] - want).max() < 1e-15
        # its moments: density rho_local, momentum rho_local * pin e_z
        assert abs(f1[:, 0, k].sum() - rho_local[0, k]) < 1e-14
        assert np.abs(c.T @ f1[:, 0, k] - [0.0, 0.0, rho_local[0, k] * pin]).max() < 1e-15
        # a reset with rho0 would differ
        assert np.abs(f1[:, 0, k] - oracle_mod.feq(1.0, [0.0, 0.0, pin])).max() > 1e-5
    # the other planes relax by Eq. 14: not the pinned equilibrium
    for z in range(1, n[2]):
        k = 3
        assert np.abs(f1[:, z, k] - oracle_mod.feq(rho_local[z, k], [0.0, 0.0, pin])).max() > 1e-6


def test_pinned_plane_drives_the_box_to_uniform_flow(oracle_mod):
    n = (4, 4, 16)
    pin = 0.01
    p = lparams(n, pin_vn=pin, tau=1.0)
    ch = oracle_mod.Channel(p)
    ch.step(3000)
    u = ch.read(oracle_mod.FIELD_U)
    assert np.abs(u[2] - pin).max() < 1e-8
    assert np.abs(u[:2]).max() < 1e-12


def momentum(oracle_mod, fstar):
    c, _, _ = oracle_mod.lattice()
    return c.T.astype(np.float64) @ fstar.sum(1)


def test_momentum_budget_of_one_pass(oracle_mod):
    n = (6, 5, 7)
    ncell = n[0] * n[1] * n[2]
    for body in ([0.0, 0.0, 0.0], [2e-6, -1e-6, 3e-6]):
        p = lparams(n, body_force=body, init_vn=[0.004, -0.002, 0.01])
        ch = oracle_mod.Channel(p)
        f0 = ch.read(oracle_mod.FIELD_FSTAR) * inputs.perturbed_equilibrium(ncell, 31, 1e-2)
        ch.write(oracle_mod.FIELD_FSTAR, f0)
        F = inputs.random_field((3, ncell), 32, 1e-4)
        ch.write(oracle_mod.FIELD_FORCE, F)
        p0 = momentum(oracle_mod, f0)
        ch.run_phases(oracle_mod.PHASE_LBM)
        p1 = momentum(oracle_mod, ch.read(oracle_mod.FIELD_FSTAR))
        want = F.sum(1) + ncell * np.asarray(body)
        assert np.abs(F.sum(1)).min() > 1e-4  # a force budget well above round-off
        assert np.abs((p1 - p0) - want).max() < 1e-13


def vector_area(x, nxt):
    return 0.5 * np.cross(x, x[nxt]).sum(0)


def test_friction_reaction_balances_the_ring_impulse(oracle_mod):
    """form 1: the normal fluid gains what the vortex impulse loses"""
    n = (32, 32, 32)
    for T, normal, R in ((1.9, (0.3, 0.2, 0.93), 6.0), (1.6, (-0.5, 0.1, 0.4), 7.5)):
        p = configs.base_params(n, (0, 0, 0), T, force_form=1, max_points=256)
        xyz, nxt = inputs.ring((16.0, 15.0, 17.0), normal, R, npts=int(round(2 * math.pi * R / 0.8)))
        ch = oracle_mod.Channel(p)
        ch.seed(xyz, nxt)
        x0 = ch.read(oracle_mod.FIELD_POS)
        ch.run_phases(oracle_mod.PHASE_VFM)
        x1 = ch.read(oracle_mod.FIELD_POS)
        nx = ch.read(oracle_mod.FIELD_NEXT)
        dA = vector_area(x1, nx) - vector_area(x0, nx)  # one step: dt = 1
        F = ch.read(oracle_mod.FIELD_FORCE).sum(1)
        want = -p["rho_s_over_rho_n"] * p["rho0"] * p["kappa"] * dA
        assert np.linalg.norm(F - want) < 1e-3 * np.linalg.norm(want)


def chord_ring(chords, center):
    """Points on a circle whose consecutive chords have the given lengths."""
    chords = np.asarray(chords, np.float64)
    lo, hi = chords.max() / 2 + 1e-9, 1e3
    for _ in range(200):
        R = 0.5 * (lo + hi)
        tot = (2 * np.arcsin(chords / (2 * R))).sum()
        if tot > 2 * math.pi:
            lo = R
        else:
            hi = R
    th = np.concatenate([[0.0], np.cumsum(2 * np.arcsin(chords / (2 * R)))[:-1]])
    xyz = np.c_[center[0] + R * np.cos(th), center[1] + R * np.sin(th), np.full(len(th), center[2])]
    nxt = ((np.arange(len(th)) + 1) % len(th)).astype(np.int32)
    return xyz, nxt


# MurmurHash3 32-bit finaliser of the point indices that meet below
FMIX32 = {5: 0xCC0D53CD, 6: 0x5CEB4D08, 11: 0x93A0FE04, 12: 0x7C88AD73, 13: 0x95BB7D92,
          20: 0xD24B0921, 21: 0xEA126165}


def test_merge_priority_of_neighbouring_candidates(oracle_mod):
    # segment k runs from point k to k + 1; short runs make points 5, 6 (pair),
    # 11, 12, 13 (triple) and 20, 21 (pair) the only merge candidates
    chords = np.full(30, 0.8)
    chords[[4, 5, 6]] = 0.3
    chords[[10, 11, 12, 13]] = 0.25
    chords[[19, 20, 21]] = 0.3
    xyz, nxt = chord_ring(chords, (10.0, 10.0, 10.0))
    p = configs.base_params((20, 20, 20), (0, 0, 0), 1.9, couple=0, max_points=256)
    ch = oracle_mod.Channel(p)
    ch.seed(xyz, nxt)
    ch.run_phases(oracle_mod.PHASE_REMESH)
    # a candidate goes unless a candidate neighbour has the larger hash
    cands = [5, 6, 11, 12, 13, 20, 21]
    removed = [i for i in cands
               if not any(j in cands and FMIX32[j] > FMIX32[i] for j in (i - 1, i + 1))]
    assert removed == [5, 11, 13, 21]
    keep = [i for i in range(30) if i not in removed]
    x1 = ch.read(oracle_mod.FIELD_POS)
    assert ch.n_points() == len(keep)
    assert np.array_equal(x1, xyz[keep])
    assert np.array_equal(ch.read(oracle_mod.FIELD_NEXT), (np.arange(len(keep)) + 1) % len(keep))
    assert ch.stats()[6] == 4  # merges counted
    # (the reversed order would have removed 6, 12 and 20 instead)
