"""Wall-bound filaments on the GPU vs the oracle (Sec. IV: lines bound to the
solid walls of the closed channel).

Bit-exact: the seeded state (open ends moved onto wall bounds), remeshing and
reconnection with open lines, including the wall-contact cuts.  Within the
float tolerance of the other advance tests: the stage-1 velocity and the
displacement of one filament advance with pinned ends (whose wall-normal
velocity must be exactly zero on both sides), the stand-alone Biot-Savart
entry point on open lines, and one whole coupled step of the closed channel
seeded with wall-bound lines and rings."""
import numpy as np
import pytest

from gpu_util import pair, rel_l2

pytestmark = pytest.mark.gpu


def wparams(n, wall, **kw):
    from paper_2108_04435_gb300 import configs
    kw.setdefault("max_points", 16384)
    return configs.base_params(n, wall, 1.9, **kw)


def wall_tangle(n, wall, seed, jitter=0.25, lines=6, rings=10, spacing=0.8, amp=2.0, touch=3):
    """Jittered wall lines and rings, the first ``touch`` rings moved against
    the low z wall; points pushed past a wall are clamped onto its bound at
    seeding, so the first reconnection pass cuts their loops there."""
    from paper_2108_04435_gb300 import inputs
    L = inputs.wall_lines(n, lines, seed, amp=amp, spacing=spacing)
    r_max = min(7.0, min(n[a] for a in range(3) if wall[a]) / 2.0 - 3.0)
    rx, rn = inputs.random_rings(n, wall, rings, 2.0, r_max, seed + 1, spacing=spacing, min_sep=0.0)
    rx = rx.copy()
    starts = [k for k in range(len(rn)) if k == 0 or rn[k - 1] != k]  # first point of each ring
    for r0 in starts[:touch]:
        r1 = r0
        while rn[r1] != r0:
            r1 += 1
        rx[r0:r1 + 1, 2] += -0.3 - rx[r0:r1 + 1, 2].min()
    xyz, nxt = inputs.concat([L, (rx, rn)])
    rng = np.random.default_rng(seed + 100)
    xyz = xyz + jitter * rng.uniform(-1, 1, xyz.shape)
    for a in range(3):
        if wall[a]:
            xyz[:, a] = np.clip(xyz[:, a], -0.45, n[a] - 0.55)
        else:
            xyz[:, a] = np.mod(xyz[:, a], n[a])
    return xyz, nxt


def assert_same_points(g, r):
    import oracle
    from paper_2108_04435_gb300 import vlb
    assert g.n_points() == r.n_points()
    assert np.array_equal(g.read(vlb.FIELD_NEXT), r.read(oracle.FIELD_NEXT))
    assert np.array_equal(g.read(vlb.FIELD_POS), r.read(oracle.FIELD_POS))
    sg, sr = g.stats(), r.stats()
    assert np.array_equal(sg[5:9], sr[5:9]), (sg[5:9], sr[5:9])
    assert sg[13] == sr[13], (sg[13], sr[13])


def test_seed_moves_ends_onto_bounds():
    n, wall = (24, 20, 32), (1, 1, 1)
    xyz, nxt = wall_tangle(n, wall, 0)
    g, r = pair(wparams(n, wall, couple=0), xyz, nxt)
    assert_same_points(g, r)


@pytest.mark.parametrize("spacing,seed", [(1.02, 0), (0.45, 1), (0.8, 2)])
def test_remesh_open_lines_bit_exact(spacing, seed):
    import oracle
    from paper_2108_04435_gb300 import vlb
    n, wall = (24, 20, 32), (1, 1, 1)
    xyz, nxt = wall_tangle(n, wall, seed, spacing=spacing)
    g, r = pair(wparams(n, wall, couple=0), xyz, nxt)
    for _ in range(3):
        g.run_phases(vlb.PHASE_REMESH)
        r.run_phases(oracle.PHASE_REMESH)
        assert_same_points(g, r)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_reconnect_and_contact_bit_exact(seed):
    import oracle
    from paper_2108_04435_gb300 import vlb
    n, wall = (16, 16, 24), (1, 0, 1)
    xyz, nxt = wall_tangle(n, wall, seed, jitter=0.35, lines=8, rings=12)
    g, r = pair(wparams(n, wall, couple=0), xyz, nxt)
    for _ in range(2):
        g.run_phases(vlb.PHASE_RECONNECT)
        r.run_phases(oracle.PHASE_RECONNECT)
        assert_same_points(g, r)
    assert r.stats()[13] > 0  # the case exercises the contact cut


def test_hand_cases():
    """The oracle's hand-worked cases (contact cut of an octagon; two
    antiparallel wall lines reconnecting) give the same arrays on the GPU."""
    import oracle
    from paper_2108_04435_gb300 import inputs, vlb
    from test_oracle_walls import antiparallel_lines, octagon_touching, wparams as owp
    p = owp()
    for xyz, nxt in (octagon_touching(p), antiparallel_lines(p)):
        g, r = pair(p, xyz, nxt)
        g.run_phases(vlb.PHASE_RECONNECT)
        r.run_phases(oracle.PHASE_RECONNECT)
        assert_same_points(g, r)
    lo, hi = -0.5 + 0.5 * p["dxi_min"], p["n"][2] - 0.5 - 0.5 * p["dxi_min"]
    z = [lo, lo + 1.2, 1.85, 2.65, 3.45, 4.25, hi]
    g, r = pair(p, *inputs.open_line(np.c_[np.full(7, 4.0), np.full(7, 5.0), z]))
    g.run_phases(vlb.PHASE_REMESH)
    r.run_phases(oracle.PHASE_REMESH)
    assert_same_points(g, r)


@pytest.mark.parametrize("couple", [0, 1])
def test_advance_with_pinned_ends(couple):
    import oracle
    from paper_2108_04435_gb300 import vlb
    n, wall = (24, 20, 32), (1, 1, 1)
    xyz, nxt = wall_tangle(n, wall, 5, jitter=0.05)
    p = wparams(n, wall, couple=couple, heater_vn=0.01, init_vn=[0.0, 0.0, 0.01])
    g, r = pair(p, xyz, nxt)
    p0 = r.read(oracle.FIELD_POS)
    nx = r.read(oracle.FIELD_NEXT)
    g.run_phases(vlb.PHASE_LBM | vlb.PHASE_VFM)
    r.run_phases(oracle.PHASE_LBM | oracle.PHASE_VFM)
    vg, vr = g.read(vlb.FIELD_VEL), r.read(oracle.FIELD_VEL)
    assert rel_l2(vg, vr) < 1e-5
    pg, pr = g.read(vlb.FIELD_POS), r.read(oracle.FIELD_POS)
    assert rel_l2(pg - p0, pr - p0) < 1e-5
    has_pred = np.zeros(len(nx), bool)
    has_pred[nx[nx >= 0]] = True
    ends = np.where((nx < 0) | ~has_pred)[0]
    assert len(ends) >= 12
    lo = -0.5 + 0.5 * p["dxi_min"]
    for k in ends:  # each end keeps its wall coordinate exactly, with zero normal velocity
        on = [a for a in range(3) if wall[a] and (p0[k, a] <= lo or p0[k, a] >= n[a] - 0.5 - 0.5 * p["dxi_min"])]
        assert on
        a = on[0]
        assert vg[k, a] == 0.0 and vr[k, a] == 0.0
        assert pg[k, a] == p0[k, a] and pr[k, a] == p0[k, a]
    if couple:
        assert rel_l2(g.read(vlb.FIELD_FORCE), r.read(oracle.FIELD_FORCE)) < 1e-5


def test_biot_savart_entry_point_open_lines():
    import oracle
    from test_gpu_vfm import _bs_gpu
    n, wall = (24, 20, 32), (1, 1, 1)
    xyz, nxt = wall_tangle(n, wall, 7, jitter=0.05)
    p = wparams(n, wall, couple=0)
    r = oracle.Channel(p)
    r.seed(xyz, nxt)
    _, vbs = r.point_velocity()
    got = _bs_gpu(p, r.read(oracle.FIELD_POS), r.read(oracle.FIELD_NEXT))
    assert rel_l2(got, vbs) < 1e-5


def test_channel_lines_one_step():
    """The closed channel seeded as in Sec. IV (four wall lines, two rings)."""
    import oracle
    from paper_2108_04435_gb300 import configs
    from test_gpu_step import compare_step
    p, xyz, nxt = configs.config("channel64x64x256_lines")
    g, r = pair(p, xyz, nxt)
    x0 = r.read(oracle.FIELD_POS)
    g.step(1)
    r.step(1)
    pg, pr = compare_step(g, r, xyz, p["n"], p["wall"])
    if len(pr) == len(x0):
        assert rel_l2(pg - x0, pr - x0) < 1e-5


@pytest.mark.parametrize("wall", [(1, 1, 1), (1, 0, 1)], ids=["walls-all", "walls-xz"])
def test_advance_with_wall_images(wall):
    """The boundary-induced velocity from wall images (wall_images = 1): the
    Biot-Savart sources then include the mirror image of every segment across
    each solid face, and a pinned end skips its own segment's image."""
    import oracle
    from paper_2108_04435_gb300 import vlb
    n = (24, 20, 32)
    xyz, nxt = wall_tangle(n, wall, 6, jitter=0.05)
    p = wparams(n, wall, couple=1, wall_images=1, heater_vn=0.01, init_vn=[0.0, 0.0, 0.01])
    g, r = pair(p, xyz, nxt)
    p0 = r.read(oracle.FIELD_POS)
    g.run_phases(vlb.PHASE_LBM | vlb.PHASE_VFM)
    r.run_phases(oracle.PHASE_LBM | oracle.PHASE_VFM)
    assert rel_l2(g.read(vlb.FIELD_VEL), r.read(oracle.FIELD_VEL)) < 1e-5
    assert rel_l2(g.read(vlb.FIELD_POS) - p0, r.read(oracle.FIELD_POS) - p0) < 1e-5
    assert rel_l2(g.read(vlb.FIELD_FORCE), r.read(oracle.FIELD_FORCE)) < 1e-5
    # the images change the motion: the same state without them moves differently
    q = dict(p, wall_images=0)
    r0 = oracle.Channel(q)
    r0.seed(xyz, nxt)
    r0.run_phases(oracle.PHASE_LBM | oracle.PHASE_VFM)
    assert rel_l2(r0.read(oracle.FIELD_VEL), r.read(oracle.FIELD_VEL)) > 1e-3


def test_channel_lines_with_images_steps():
    """Ten whole steps of the Sec. IV seed with wall images, GPU vs oracle."""
    import oracle
    from paper_2108_04435_gb300 import configs, vlb
    from test_gpu_step import compare_step
    p, xyz, nxt = configs.config("channel64x64x256_lines")
    p = dict(p, wall_images=1)
    g, r = pair(p, xyz, nxt)
    g.step(10)
    r.step(10)
    compare_step(g, r, xyz, p["n"], p["wall"], tol=2e-5, line_tol=1e-7)
