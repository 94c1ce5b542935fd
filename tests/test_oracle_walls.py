"""Pins of the oracle's wall-bound filaments (Sec. IV: vortex lines bound to
the solid walls of the closed channel).

Readings pinned here: an open end is pinned to the wall whose clamp bound it
touches; its missing neighbour is the mirror image of the present one across
that wall; its wall-normal velocity is zero; a point with both neighbours that
touches a wall's bound cuts its line there (it is deleted and its neighbours
become pinned ends on that bound).  The cases:
- seeding accepts closed loops and open lines only, and only with the open
  ends near a wall, which it moves onto the wall's clamp bound;
- a straight line spanning the channel has s' = e_z, s'' = 0 and no local or
  Biot-Savart velocity; under a uniform applied flow its points move with it
  except the ends, which do not leave the walls; its length is the span;
- a half circle standing on a wall has, at its pinned ends, the geometry of
  the full circle (the mirror image continues it exactly);
- hand-worked cases: a ring touching a wall is cut into one open line; a
  5-point ring cut the same way leaves a 4-point line, which is deleted; a long
  segment at an end is split at its midpoint; two antiparallel wall-bound lines
  reconnect into two U-shaped lines;
- a ring driven into a wall by its own motion ends up as a line pinned on that
  wall, and all ends stay on wall bounds throughout;
- wall images (the boundary-induced velocity v_s,b): a line parallel to the
  walls moves at the closed-form velocity of its two image lines; a half
  circle standing on a wall plus its images is the full circle, ends included;
  a line perpendicular to the walls gets nothing from its collinear images.
"""
import numpy as np
import pytest

from paper_2108_04435_gb300 import configs, inputs


def wparams(n=(12, 12, 6), wall=(0, 0, 1), **kw):
    kw.setdefault("couple", 0)
    kw.setdefault("max_points", 1024)
    return configs.base_params(n, wall, 1.9, **kw)


def bounds(p, axis):
    lo = -0.5 + 0.5 * p["dxi_min"]
    hi = p["n"][axis] - 0.5 - 0.5 * p["dxi_min"]
    return lo, hi


def chains(nxt):
    """Components as index lists: open lines from their first point, then loops."""
    n = len(nxt)
    has_pred = np.zeros(n, bool)
    for k in range(n):
        if nxt[k] >= 0:
            has_pred[nxt[k]] = True
    seen = np.zeros(n, bool)
    out = []
    for s in [k for k in range(n) if not has_pred[k]] + list(range(n)):
        if seen[s]:
            continue
        comp, j = [], s
        while j >= 0 and not seen[j]:
            seen[j] = True
            comp.append(j)
            j = nxt[j]
        out.append(comp)
    return out


def ends_on_bounds(p, pos, nxt):
    """Every open end lies on some wall's clamp bound."""
    has_pred = np.zeros(len(nxt), bool)
    has_pred[nxt[nxt >= 0]] = True
    for k in range(len(nxt)):
        if nxt[k] >= 0 and has_pred[k]:
            continue
        ok = False
        for a in range(3):
            if p["wall"][a]:
                lo, hi = bounds(p, a)
                ok |= pos[k, a] <= lo or pos[k, a] >= hi
        if not ok:
            return False
    return True


def test_seed_rules(oracle_mod):
    p = wparams()
    line = inputs.wall_line((4.0, 4.0, 0.2), (4.0, 4.0, 4.9))
    ch = oracle_mod.Channel(p)
    ch.seed(*line)
    pos = ch.read(oracle_mod.FIELD_POS)
    lo, hi = bounds(p, 2)
    assert pos[0, 2] == lo and pos[-1, 2] == hi  # ends moved onto the bounds
    assert np.array_equal(pos[1:-1], line[0][1:-1])
    # an end farther than dxi_max from every wall
    far = inputs.wall_line((4.0, 4.0, 0.2), (4.0, 4.0, 3.0))
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Channel(p).seed(*far)
    # open lines need walls
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Channel(wparams(wall=(0, 0, 0))).seed(*line)
    # an isolated point; a point with two predecessors
    xyz = np.array([[4.0, 4.0, 0.0]])
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Channel(p).seed(xyz, np.array([-1], np.int32))
    xyz, nxt = inputs.ring((6.0, 6.0, 2.5), (0, 0, 1), 1.5, npts=12)
    nxt = nxt.copy()
    nxt[3] = 5
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Channel(p).seed(xyz, nxt)


def test_straight_spanning_line(oracle_mod):
    """Collinear segments: no local term, no Biot-Savart velocity; the applied
    flow V_s e_z moves the interior points along the line and not the ends."""
    vn = 0.02
    p = wparams(n=(12, 12, 16), init_vn=[0.0, 0.0, vn])
    ch = oracle_mod.Channel(p)
    ch.seed(*inputs.wall_line((5.3, 6.1, 0.0), (5.3, 6.1, 15.0), spacing=0.9))
    sp, spp, dxi, lia = ch.geometry()
    assert np.abs(sp - [0.0, 0.0, 1.0]).max() < 1e-15
    assert np.abs(spp).max() < 1e-12 and np.abs(lia).max() < 1e-12
    lo, hi = bounds(p, 2)
    assert abs(ch.line_length() - (hi - lo)) < 1e-12
    vel, vbs = ch.point_velocity()
    assert np.abs(vbs).max() < 1e-14
    Vs = ch.read(oracle_mod.FIELD_PLANE_VS)[0]
    assert Vs != 0.0
    assert np.abs(vel[1:-1] - [0.0, 0.0, Vs]).max() < 1e-15
    assert np.all(vel[[0, -1]] == 0.0)
    ch.run_phases(oracle_mod.PHASE_VFM)
    pos = ch.read(oracle_mod.FIELD_POS)
    assert pos[0, 2] == lo and pos[-1, 2] == hi


@pytest.mark.parametrize("m", [9, 13])
def test_half_circle_on_wall_has_full_circle_geometry(oracle_mod, m):
    """A half circle of m points standing on the z-low wall (centre on the
    wall plane z = -1/2): the mirror image of each end's neighbour is the
    circle's next point, so the ends see the geometry of the full 2(m-1)-gon."""
    R = 2.5
    p = wparams(n=(16, 16, 8), dxi_min=1e-9, dxi_max=1.2)
    th = np.pi * np.arange(m) / (m - 1)
    xyz = np.c_[8.0 + R * np.cos(th), np.full(m, 8.0), -0.5 + R * np.sin(th)]
    xyz[[0, -1], 2] = -0.5 + 1e-10
    ch = oracle_mod.Channel(p)
    ch.seed(*inputs.open_line(xyz))
    sp, spp, dxi, lia = ch.geometry()
    mid = m // 2
    for e in (0, m - 1):
        assert abs(np.linalg.norm(spp[e]) - np.linalg.norm(spp[mid])) < 1e-8
        assert abs(np.linalg.norm(lia[e]) - np.linalg.norm(lia[mid])) < 1e-9
        assert abs(np.linalg.norm(sp[e]) - np.linalg.norm(sp[mid])) < 1e-8
    # the end's curvature points to the centre, its tangent along the wall normal
    t0, t1 = sp[0] / np.linalg.norm(sp[0]), sp[-1] / np.linalg.norm(sp[-1])
    assert np.abs(t0 - [0, 0, 1]).max() < 1e-8 and np.abs(t1 - [0, 0, -1]).max() < 1e-8
    assert spp[0, 0] < 0 and spp[-1, 0] > 0
    # the ends represent half a segment
    chord = 2 * R * np.sin(np.pi / (2 * (m - 1)))
    assert abs(dxi[0] - 0.5 * chord) < 1e-8 and abs(dxi[mid] - chord) < 1e-12


def octagon_touching(p, k_touch=6):
    """An 8-point ring in the x-z plane whose point 6 (the lowest) lies below
    the z-low bound, so seeding clamps it onto the bound."""
    R = 1.2
    th = 2 * np.pi * np.arange(8) / 8
    xyz = np.c_[6.0 + R * np.cos(th), np.full(8, 6.0), 0.95 + R * np.sin(th)]
    assert np.argmin(xyz[:, 2]) == k_touch
    return xyz, ((np.arange(8) + 1) % 8).astype(np.int32)


def test_contact_cut_by_hand(oracle_mod):
    """Point 6 touches the low wall: it is deleted, 5 becomes the last point
    and 7 the first, both moved onto the bound; after compaction old 7 is
    new 6: next = [1, 2, 3, 4, 5, -1, 0]."""
    p = wparams()
    xyz, nxt = octagon_touching(p)
    ch = oracle_mod.Channel(p)
    ch.seed(xyz, nxt)
    lo, _ = bounds(p, 2)
    assert ch.read(oracle_mod.FIELD_POS)[6, 2] == lo
    ch.run_phases(oracle_mod.PHASE_RECONNECT)
    assert ch.n_points() == 7
    assert ch.read(oracle_mod.FIELD_NEXT).tolist() == [1, 2, 3, 4, 5, -1, 0]
    pos = ch.read(oracle_mod.FIELD_POS)
    want = xyz[[0, 1, 2, 3, 4, 5, 7]].copy()
    want[[5, 6], 2] = lo
    assert np.array_equal(pos, want)
    st = ch.stats()
    assert st[13] == 1 and st[7] == 0


def test_small_open_line_deleted(oracle_mod):
    """A pentagon touching the wall is cut into a 4-point line, which is
    deleted in the same pass."""
    p = wparams()
    R = 0.7
    th = -np.pi / 2 + 2 * np.pi * np.arange(5) / 5
    xyz = np.c_[6.0 + R * np.cos(th), np.full(5, 6.0), -0.2 + R + R * np.sin(th)]
    ch = oracle_mod.Channel(p)
    ch.seed(xyz, ((np.arange(5) + 1) % 5).astype(np.int32))
    ch.run_phases(oracle_mod.PHASE_RECONNECT)
    st = ch.stats()
    assert ch.n_points() == 0 and st[13] == 1 and st[8] == 4


def test_split_at_an_end(oracle_mod):
    """Segment 0 -> 1 of a straight wall-bound line is 1.2 > dxi_max: its
    midpoint (the arc correction vanishes: the end's image is collinear) is
    appended as point 7; the 0.9-long last segment stays; no point is removed."""
    p = wparams()
    lo, hi = bounds(p, 2)
    z = [lo, lo + 1.2, 1.85, 2.65, 3.45, 4.25, hi]
    ch = oracle_mod.Channel(p)
    ch.seed(*inputs.open_line(np.c_[np.full(7, 4.0), np.full(7, 5.0), z]))
    ch.run_phases(oracle_mod.PHASE_REMESH)
    assert ch.n_points() == 8
    assert ch.read(oracle_mod.FIELD_NEXT).tolist() == [7, 2, 3, 4, 5, 6, -1, 1]
    pos = ch.read(oracle_mod.FIELD_POS)
    assert np.array_equal(pos[7], [4.0, 5.0, lo + 0.5 * (z[1] - lo)])
    assert pos[0, 2] == lo and pos[6, 2] == hi


def antiparallel_lines(p):
    lo, hi = bounds(p, 2)
    z = lo + (hi - lo) * np.arange(8) / 7
    A = np.c_[np.full(8, 4.0), np.full(8, 4.0), z]
    B = np.c_[np.full(8, 6.0), np.full(8, 4.0), z[::-1]]
    B[[3, 4, 5], 0] = 4.5  # B3, B4, B5 bent to 0.5 from A4, A3, A2
    return inputs.concat([inputs.open_line(A), inputs.open_line(B)])


def test_antiparallel_wall_lines_reconnect_by_hand(oracle_mod):
    """Segments of 0.757 along z; B's points 3-5 sit 0.5 from A's 4-2.  Mutual
    pairs (A2,B5), (A3,B4), (A4,B3), all at d^2 = 0.25, taken in order of i.
    For (A2,B5) the best exchange is on A2->A3 and B4->B5 (gain
    2(0.757) - 2(0.5) > 0); the other two pairs touch A3 and are skipped.
    Result: A2 -> B5 and B4 -> A3, i.e. two U-shaped lines, one on each wall:
    A0 A1 A2 B5 B6 B7 and B0 .. B4 A3 .. A7."""
    p = wparams()
    xyz, nxt = antiparallel_lines(p)
    ch = oracle_mod.Channel(p)
    ch.seed(xyz, nxt)
    L0 = ch.line_length()
    ch.run_phases(oracle_mod.PHASE_RECONNECT)
    want = nxt.copy()
    want[2] = 8 + 5
    want[8 + 4] = 3
    assert ch.read(oracle_mod.FIELD_NEXT).tolist() == want.tolist()
    comps = chains(want)
    assert sorted(len(c) for c in comps) == [6, 10]
    seg = np.linalg.norm(xyz[3] - xyz[2])
    assert abs((L0 - ch.line_length()) - 2 * (seg - 0.5)) < 1e-12
    assert ch.stats()[7] == 1


def test_ring_driven_into_wall_becomes_pinned_line(oracle_mod):
    """A ring moving towards the low z wall under its own induction (normal
    -z) is cut when it reaches the wall; from then on its line ends stay on
    the wall's bound and every component keeps at least five points."""
    p = wparams(n=(16, 16, 12))
    xyz, nxt = inputs.ring((8.0, 8.0, 3.0), (0.0, 0.3, -1.0), 3.0)
    ch = oracle_mod.Channel(p)
    ch.seed(xyz, nxt)
    lo, _ = bounds(p, 2)
    for _ in range(60):
        ch.step(1)
        pos, nx = ch.read(oracle_mod.FIELD_POS), ch.read(oracle_mod.FIELD_NEXT)
        assert ends_on_bounds(p, pos, nx)
        assert all(len(c) >= 5 for c in chains(nx))
        assert pos[:, 2].min() >= lo
    st = ch.stats()
    assert st[13] >= 1
    ends = [k for k in range(len(nx)) if nx[k] < 0]
    assert len(ends) >= 1 and all(pos[k, 2] == lo for k in ends)


def test_images_of_a_line_parallel_to_the_walls(oracle_mod):
    """A straight line along the periodic z axis between two x walls sees its
    two images (antiparallel lines at twice its distance to each wall): it
    moves along y at g(D_hi) - g(D_lo), with g the velocity of the finite image
    line the minimum image leaves (m segments of L/m, odd m: from (m+1)L/(2m)
    below the target to (m-1)L/(2m) above)."""
    nx, L, m = 16, 32, 41
    x0, y0 = 4.3, 7.0
    p = wparams(n=(nx, 16, L), wall=(1, 0, 0), wall_images=1)
    z = L * np.arange(m) / m
    xyz = np.c_[np.full(m, x0), np.full(m, y0), z]
    nxt = ((np.arange(m) + 1) % m).astype(np.int32)
    ch = oracle_mod.Channel(p)
    ch.seed(xyz, nxt)
    _, vbs = ch.point_velocity()
    a, b = (m + 1) * L / (2 * m), (m - 1) * L / (2 * m)

    def g(D):
        return p["kappa"] / (4 * np.pi * D) * (a / np.hypot(a, D) + b / np.hypot(b, D))

    D_lo, D_hi = 2 * (x0 + 0.5), 2 * (nx - 0.5 - x0)
    vy = g(D_hi) - g(D_lo)
    assert vy < 0  # nearer to the low wall: pulled along -y
    assert np.abs(vbs[:, 1] - vy).max() < 1e-12 * abs(vy)
    assert np.abs(vbs[:, [0, 2]]).max() < 1e-15
    # without images the straight line has no velocity at all
    ch0 = oracle_mod.Channel(wparams(n=(nx, 16, L), wall=(1, 0, 0)))
    ch0.seed(xyz, nxt)
    assert np.abs(ch0.point_velocity()[1]).max() < 1e-15


@pytest.mark.parametrize("m", [9, 13])
def test_half_circle_and_its_image_are_the_full_circle(oracle_mod, m):
    """A half circle standing on a wall plus its images is the full circle:
    every point, the pinned ends included, gets the full circle's Biot-Savart
    velocity.  At an end this needs the exclusion rule: the image of the end's
    own segment is the full circle's other adjacent segment."""
    R = 2.5
    # the far z wall sits 1024 cells away: its image of the open arc adds
    # ~ kappa l / d^2 ~ 1.5e-8 (1e-6 relative); a wrong exclusion at the ends
    # would be off by the adjacent segment's ~1e-2
    p = wparams(n=(16, 16, 1024), dxi_min=1e-9, dxi_max=1.2, wall_images=1)
    th = np.pi * np.arange(m) / (m - 1)
    half = np.c_[8.0 + R * np.cos(th), np.full(m, 8.0), -0.5 + R * np.sin(th)]
    half[[0, -1], 2] = -0.5 + 1e-10
    ch = oracle_mod.Channel(p)
    ch.seed(*inputs.open_line(half))
    _, v_half = ch.point_velocity()
    M = 2 * (m - 1)
    thf = 2 * np.pi * np.arange(M) / M
    full = np.c_[32.0 + R * np.cos(thf), np.full(M, 32.0), 32.0 + R * np.sin(thf)]
    cf = oracle_mod.Channel(wparams(n=(64, 64, 64), wall=(0, 0, 0)))
    cf.seed(full, ((np.arange(M) + 1) % M).astype(np.int32))
    _, v_full = cf.point_velocity()
    assert np.abs(v_half - v_full[:m]).max() < 1e-5 * np.abs(v_full).max()


def test_images_leave_a_spanning_line_still(oracle_mod):
    """The images of a line perpendicular to the walls are collinear with it."""
    p = wparams(n=(12, 12, 16), wall_images=1)
    ch = oracle_mod.Channel(p)
    ch.seed(*inputs.wall_line((5.3, 6.1, 0.0), (5.3, 6.1, 15.0), spacing=0.9))
    _, vbs = ch.point_velocity()
    assert np.abs(vbs).max() < 1e-15
