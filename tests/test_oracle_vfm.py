"""Pins of the oracle's vortex-filament pieces (Sec. II.A, Eqs. 3-4, 10-11, 15).

- the straight-segment Biot-Savart closed form against Gauss-Legendre
  quadrature of the Eq. 3 integrand, and the infinite line kappa/(2 pi d);
- geometry of a regular N-gon (exact curvature 1/R, exact perimeter);
- self-induced ring speed kappa/(4 pi R)(ln(8R/a) - 1/4) (the solid-core
  constant that Schwarz's cutoff reproduces) and its direction;
- mutual-friction shrink d(R^2)/dt = -2 alpha kappa/(4 pi)(ln(8R/a) - 1/4)
  (the form of Eq. 15 with the local-induction speed);
- the two friction terms of Eq. 4 on a ring at rest in the normal fluid:
  alpha' slows it by 1 - alpha'|s'|^2, alpha moves it inward at alpha|s'||v_s|;
- coupling slows the shrink (Sec. III.A, Fig. 2d);
- the 2-point delta interpolation (Eq. 11) reproduces affine fields and
  reaches one cell per axis, and spreading is its exact adjoint with
  partition of unity;
- periodic translation invariance: rings shifted and wrapped across the
  faces of a periodic box move exactly as before (the minimum image);
- the RK4 integration of Eq. 4 converges at fourth order in the sub-step
  (a first-order-consistent slip in the stage weights passes the ring-speed
  and shrink-rate pins but fails this one).
"""
import numpy as np
import pytest

from paper_2108_04435_gb300 import configs, inputs


def vparams(n=(64, 64, 64), wall=(0, 0, 0), **kw):
    kw.setdefault("couple", 0)
    kw.setdefault("max_points", 1024)
    return configs.base_params(n, wall, 1.9, **kw)


@pytest.mark.parametrize("seed", range(5))
def test_segment_closed_form_vs_quadrature(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    kappa = 0.157
    r = rng.uniform(-1, 1, 3)
    s1 = rng.uniform(-3, 3, 3)
    s2 = s1 + rng.uniform(-2, 2, 3)
    got = oracle_mod.segment_velocity(r, s1, s2, kappa)
    x, wq = np.polynomial.legendre.leggauss(64)
    t = 0.5 * (x + 1.0)
    d = s2 - s1
    pts = s1[None, :] + t[:, None] * d[None, :]
    R = pts - r[None, :]
    integrand = np.cross(R, d[None, :]) / np.linalg.norm(R, axis=1)[:, None] ** 3
    ref = kappa / (4 * np.pi) * 0.5 * (wq[:, None] * integrand).sum(axis=0)
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_straight_line_telescopes_and_limits(oracle_mod):
    kappa, d = 0.157, 0.7
    r = np.zeros(3)
    L = 4000.0
    one = oracle_mod.segment_velocity(r, [-L, d, 0.0], [L, d, 0.0], kappa)
    xs = np.linspace(-L, L, 81)
    many = sum(oracle_mod.segment_velocity(r, [a, d, 0.0], [b, d, 0.0], kappa) for a, b in zip(xs[:-1], xs[1:]))
    assert np.abs(one - many).max() < 1e-8 * np.abs(one).max()
    # infinite line along +x at y = d: v = -kappa/(2 pi d) z
    assert abs(one[2] / (-kappa / (2 * np.pi * d)) - 1.0) < 1e-6
    assert abs(one[0]) < 1e-18 and abs(one[1]) < 1e-18


@pytest.mark.parametrize("N,R", [(48, 8.0), (64, 8.0), (31, 5.0)])
def test_ngon_geometry(oracle_mod, N, R):
    ch = oracle_mod.Channel(vparams())
    c = np.array([32.0, 32.0, 32.0])
    xyz, nxt = inputs.ring(c, (0, 0, 1), R, npts=N)
    ch.seed(xyz, nxt)
    sp, spp, dxi, lia = ch.geometry()
    # three-point curvature of a regular polygon is exactly 1/R, pointing to the centre
    assert np.abs(np.linalg.norm(spp, axis=1) * R - 1.0).max() < 1e-12
    toc = (c[None, :] - xyz) / R
    assert np.abs(spp * R - toc).max() < 1e-12
    assert np.abs(np.linalg.norm(sp, axis=1) - np.cos(np.pi / N)).max() < 1e-12
    assert abs(ch.line_length() - 2 * N * R * np.sin(np.pi / N)) < 1e-11
    l = 2 * R * np.sin(np.pi / N)
    assert np.abs(dxi - l).max() < 1e-12
    # local term along +z for a counter-clockwise ring
    assert (lia[:, 2] > 0).all() and np.abs(lia[:, :2]).max() < 1e-15


def test_ring_speed(oracle_mod):
    p = vparams(alpha=0.0, alpha_p=0.0)
    ch = oracle_mod.Channel(p)
    R = 8.0
    xyz, nxt = inputs.ring((32, 32, 32), (0, 0, 1), R, npts=64)
    ch.seed(xyz, nxt)
    v, vbs = ch.point_velocity()
    V = p["kappa"] / (4 * np.pi * R) * (np.log(8 * R / p["core_a"]) - 0.25)
    assert abs(v[:, 2].mean() / V - 1.0) < 0.01
    assert np.abs(v[:, :2]).max() < 1e-12 and np.ptp(v[:, 2]) < 1e-12
    # the same ring tilted: speed along its normal
    nrm = np.array([1.0, 2.0, 2.0]) / 3.0
    xyz, nxt = inputs.ring((32, 32, 32), nrm, R, npts=64)
    ch.seed(xyz, nxt)
    v, _ = ch.point_velocity()
    assert abs((v @ nrm).mean() / V - 1.0) < 0.01


@pytest.mark.parametrize("alpha,alpha_p", [(0.0, 0.2), (0.1, 0.0), (0.1, 0.2)])
def test_friction_terms_on_a_ring(oracle_mod, alpha, alpha_p):
    # Eq. 4 with v_n = 0 on a regular 64-gon ring: v_s at every point is
    # along the axis, perpendicular to s' (|s'| = cos(pi/N) for the central
    # difference, exact for a regular polygon), so s' x (s' x v_s) = -|s'|^2 v_s
    # and the alpha' term slows the ring by the factor 1 - alpha' |s'|^2
    # without moving it radially, while the alpha term s' x (-v_s) points to
    # the axis with magnitude alpha |s'| |v_s| (the ring shrinks) and leaves
    # the axial speed alone.
    def vel(a, ap):
        ch = oracle_mod.Channel(vparams(alpha=a, alpha_p=ap))
        xyz, nxt = inputs.ring((32, 32, 32), (0, 0, 1), 8.0, npts=64)
        ch.seed(xyz, nxt)
        v, _ = ch.point_velocity()
        ch.close()
        return xyz, np.asarray(v)

    xyz, v0 = vel(0.0, 0.0)
    _, v = vel(alpha, alpha_p)
    sp = np.cos(np.pi / 64)
    radial = (xyz - xyz.mean(axis=0)) / 8.0
    assert np.abs(v[:, 2] / v0[:, 2] - (1.0 - alpha_p * sp * sp)).max() < 1e-12
    assert np.abs((v * radial).sum(axis=1) / v0[:, 2] + alpha * sp).max() < 1e-12


def test_ring_carried_by_the_normal_fluid_feels_no_friction(oracle_mod):
    # A uniform normal flow w along the ring's axis sets V_s = -(rho_n/rho_s) w
    # (Eq. 18, box mean on a periodic box), so the superfluid velocity at the
    # ring is v_ring + V_s.  For w = v_ring r/(1 + r), r = rho_s/rho_n, that
    # equals w: the ring moves with the normal fluid, v_n - v_s = 0 at every
    # point, and both friction terms of Eq. 4 vanish, whatever alpha, alpha'.
    def vel(a, ap, w):
        p = vparams(alpha=a, alpha_p=ap, init_vn=[0.0, 0.0, w])
        ch = oracle_mod.Channel(p)
        xyz, nxt = inputs.ring((32, 32, 32), (0, 0, 1), 8.0, npts=64)
        ch.seed(xyz, nxt)
        v, _ = ch.point_velocity()
        ch.close()
        return np.asarray(v), p["rho_s_over_rho_n"]

    v0, r = vel(0.0, 0.0, 0.0)
    w = v0[:, 2].mean() * r / (1.0 + r)
    v, _ = vel(0.3, 0.2, w)
    assert np.abs(v - np.array([0.0, 0.0, w])).max() < 1e-12
    # the same flow with the friction off: the ring is slower than in still fluid by w/r
    vf, _ = vel(0.0, 0.0, w)
    assert np.abs(vf[:, 2] - (v0[:, 2] - w / r)).max() < 1e-12


@pytest.mark.parametrize("shift", [(13.3, 0.0, 0.0), (5.1, 17.7, 29.2), (16.0, 16.0, 16.0)])
def test_periodic_translation_invariance(oracle_mod, shift):
    # On an all-periodic box the velocity of Eq. 4 (Biot-Savart with the
    # minimum image, local term, friction) depends only on differences of
    # positions modulo the box: rings shifted and wrapped, several of them
    # then straddling a face, move exactly as before (to rounding).
    p = vparams((32, 32, 32))
    xyz, nxt = inputs.random_rings((32, 32, 32), (0, 0, 0), 6, 3.0, 6.0, 3)
    xyz, nxt = np.asarray(xyz), np.asarray(nxt)
    moved = (xyz + np.array(shift)) % 32.0
    raw = moved[nxt] - moved
    assert (np.abs(raw) > 16.0).any()  # some segment crosses a periodic face

    def run(x):
        ch = oracle_mod.Channel(p)
        ch.seed(x, nxt)
        v, _ = ch.point_velocity()
        length = ch.line_length()
        ch.close()
        return np.asarray(v), length

    v0, l0 = run(xyz)
    v1, l1 = run(moved)
    assert np.abs(v1 - v0).max() < 1e-11 * np.abs(v0).max()
    assert abs(l1 - l0) < 1e-11 * l0


def ring_radius(pos):
    c = pos.mean(axis=0)
    return np.linalg.norm(pos - c, axis=1).mean()


def test_ring_shrink_rate(oracle_mod):
    p = vparams()
    ch = oracle_mod.Channel(p)
    R0 = 8.0
    xyz, nxt = inputs.ring((32, 32, 32), (0, 0, 1), R0, npts=64)
    ch.seed(xyz, nxt)
    steps = 40
    ch.step(steps)
    R1 = ring_radius(ch.read(oracle_mod.FIELD_POS))
    Rm = 0.5 * (R0 + R1)
    slope = (R1 ** 2 - R0 ** 2) / steps
    pred = -2 * p["alpha"] * p["kappa"] / (4 * np.pi) * (np.log(8 * Rm / p["core_a"]) - 0.25)
    assert abs(slope / pred - 1.0) < 0.02


@pytest.mark.parametrize("form", [0, 1])
def test_coupling_slows_shrink(oracle_mod, form):
    """Sec. III.A: the coupled ring's R^2 falls more slowly (Fig. 2d)."""
    out = {}
    for couple in (0, 1):
        p = vparams(n=(32, 32, 32), couple=couple, force_form=form)
        ch = oracle_mod.Channel(p)
        xyz, nxt = inputs.ring((16, 16, 16), (0, 0, 1), 8.0, npts=64)
        ch.seed(xyz, nxt)
        ch.step(60)
        out[couple] = ring_radius(ch.read(oracle_mod.FIELD_POS))
    assert out[1] > out[0]


def test_interp_reproduces_affine_fields(oracle_mod):
    n = (9, 7, 8)
    p = vparams(n=n, wall=(1, 0, 1))
    ch = oracle_mod.Channel(p)
    ncell = n[0] * n[1] * n[2]
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    A = np.array([[0.1, -0.2, 0.3], [0.05, 0.07, -0.01], [-0.3, 0.2, 0.11]])
    b = np.array([0.5, -0.25, 1.0])
    X = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(float)
    U = (X @ A.T + b).T.copy()
    ch.write(oracle_mod.FIELD_ULAST, U)
    rng = np.random.default_rng(5)
    pts = np.stack([rng.uniform(0, n[0] - 1, 50), rng.uniform(0, n[1] - 1, 50), rng.uniform(0, n[2] - 1, 50)], axis=1)
    got = ch.interp(pts)
    assert np.abs(got - (pts @ A.T + b)).max() < 1e-13


def test_interp_support_is_one_cell(oracle_mod):
    # Eq. 11's 2-point delta has support |r| < 1 on each axis: a unit value at
    # one node reaches only points within one cell of it on every axis.  With
    # the affine exactness above this fixes the weights (the hat function is
    # the only kernel of that support reproducing linear fields); a 4-point
    # kernel, also affine-exact, fails here.
    n = (8, 8, 8)
    ch = oracle_mod.Channel(vparams(n=n))
    node = np.array([3, 4, 5])
    U = np.zeros((3, n[0] * n[1] * n[2]))
    U[:, node[0] + n[0] * (node[1] + n[1] * node[2])] = 1.0
    ch.write(oracle_mod.FIELD_ULAST, U)
    rng = np.random.default_rng(11)
    pts = np.concatenate([node + rng.uniform(-2.0, 2.0, (300, 3)), node + rng.uniform(-0.999, 0.999, (50, 3))])
    got = ch.interp(pts)
    near = (np.abs(pts - node) < 1.0).all(axis=1)
    assert near.sum() >= 50 and (~near).sum() >= 100
    assert (got[~near] == 0.0).all()
    assert (got[near] > 0.0).all()
    assert got[:, 0] == pytest.approx(got[:, 1], abs=0) and got[:, 0] == pytest.approx(got[:, 2], abs=0)


@pytest.mark.parametrize("wall", [(0, 0, 0), (1, 1, 1), (0, 1, 0)])
def test_spread_is_adjoint_of_interp(oracle_mod, wall):
    n = (6, 7, 5)
    p = vparams(n=n, wall=wall)
    ch = oracle_mod.Channel(p)
    ncell = n[0] * n[1] * n[2]
    rng = np.random.default_rng(7)
    U = rng.normal(size=(3, ncell))
    ch.write(oracle_mod.FIELD_ULAST, U)
    lo = np.array([-0.5 if w else 0.0 for w in wall])
    hi = np.array([n[a] - 0.5 if wall[a] else n[a] for a in range(3)])
    pts = lo + (hi - lo) * rng.uniform(0.001, 0.999, (40, 3))
    g = rng.normal(size=(40, 3))
    Iu = ch.interp(pts)
    ch.write(oracle_mod.FIELD_FORCE, np.zeros((3, ncell)))
    ch.spread(pts, g)
    Sg = ch.read(oracle_mod.FIELD_FORCE)
    assert abs((Iu * g).sum() - (U * Sg).sum()) < 1e-12
    assert np.abs(Sg.sum(axis=1) - g.sum(axis=0)).max() < 1e-12


def test_friction_reaction_total(oracle_mod):
    """The reaction spread in one step equals -(rho_s/rho_n) rho0 kappa sum(fr dxi)
    with fr = ds/dt - v_s (Eq. 10 as printed): partition of unity of Eq. 11."""
    p = vparams(n=(32, 32, 32), couple=1, init_vn=[0.0, 0.0, 0.01])
    ch = oracle_mod.Channel(p)
    xyz, nxt = inputs.ring((16, 16, 16), (0, 0, 1), 8.0, npts=64)
    ch.seed(xyz, nxt)
    v, vbs = ch.point_velocity()
    sp, spp, dxi, lia = ch.geometry()
    vs_plane = ch.read(oracle_mod.FIELD_PLANE_VS)[0]
    vs = vbs + lia
    vs[:, 2] += vs_plane
    fr = v - vs
    expect = -p["rho_s_over_rho_n"] * p["rho0"] * p["kappa"] * (fr * dxi[:, None]).sum(axis=0)
    ch.run_phases(oracle_mod.PHASE_VFM)
    F = ch.read(oracle_mod.FIELD_FORCE)
    assert np.abs(F.sum(axis=1) - expect).max() < 1e-15


def test_line_profile_of_tilted_ring(oracle_mod):
    """The profile sums to the line length; a ring in a z = const plane puts
    all its length in that plane, and a ring tilted about x spreads it over
    the planes it crosses symmetrically about its centre."""
    p = vparams(n=(32, 32, 32))
    ch = oracle_mod.Channel(p)
    xyz, nxt = inputs.ring((16, 16, 16.2), (0, 0, 1), 6.0, npts=48)
    ch.seed(xyz, nxt)
    prof = ch.read(oracle_mod.FIELD_LINE_PROFILE)
    assert abs(prof.sum() - ch.line_length()) < 1e-12
    assert abs(prof[16] - ch.line_length()) < 1e-12
    xyz, nxt = inputs.ring((16, 16, 16.0), (0, 1, 0), 6.0, npts=48)
    ch.seed(xyz, nxt)
    prof = ch.read(oracle_mod.FIELD_LINE_PROFILE)
    assert abs(prof.sum() - ch.line_length()) < 1e-12
    assert np.abs(prof[10:16][::-1] - prof[17:23]).max() < 0.2
    assert prof[:9].sum() == 0 and prof[24:].sum() == 0


def test_rk4_is_fourth_order(oracle_mod):
    # Eq. 4 integrated by classic RK4 over vfm_substeps sub-steps of a lattice
    # step: a small tilted ring under mutual friction (v_n = 0, no coupling),
    # four steps, against 64 sub-steps.  Halving the sub-step must cut the
    # error ~16x (Euler 2x, a second-order scheme 4x, wrong RK4 weights less).
    def run(sub):
        p = vparams((32, 32, 32), vfm_substeps=sub, max_points=256)
        ch = oracle_mod.Channel(p)
        xyz, nxt = inputs.ring((16.0, 16.0, 16.0), (0.3, 0.2, 1.0), 1.2, npts=10)
        ch.seed(xyz, nxt)
        for _ in range(4):
            ch.run_phases(oracle_mod.PHASE_VFM)
        x = ch.read(oracle_mod.FIELD_POS).copy()
        ch.close()
        return x

    ref = run(64)
    e = [np.abs(run(s) - ref).max() for s in (1, 2, 4)]
    assert e[0] > 1e-9  # the ring moves enough over a step for the order to show
    for a, b in zip(e, e[1:]):
        assert 12.0 < a / b < 20.0, e
