"""GPU remeshing and reconnection vs the oracle: bit-exact integer results.

From identical inputs the successor array, the point count, the counters and
the positions (old points copied, new points computed by the same FP64
expression without contraction) must be identical."""
import numpy as np
import pytest

from gpu_util import pair

pytestmark = pytest.mark.gpu


def tparams(n, wall, **kw):
    from paper_2108_04435_gb300 import configs
    kw.setdefault("couple", 0)
    kw.setdefault("max_points", 16384)
    return configs.base_params(n, wall, 1.9, **kw)


def jittered_tangle(n, wall, count, seed, jitter, spacing):
    from paper_2108_04435_gb300 import inputs
    xyz, nxt = inputs.random_rings(n, wall, count, 2.0, 9.0, seed, spacing=spacing, min_sep=0.0)
    rng = np.random.default_rng(seed + 100)
    xyz = xyz + jitter * rng.uniform(-1, 1, xyz.shape)
    for a in range(3):
        if wall[a]:
            xyz[:, a] = np.clip(xyz[:, a], 0.0, n[a] - 1.0)
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


@pytest.mark.parametrize("spacing,jitter,seed", [(1.02, 0.05, 0), (0.45, 0.05, 1), (0.8, 0.3, 2), (0.6, 0.2, 3)])
def test_remesh_bit_exact(spacing, jitter, seed):
    import oracle
    from paper_2108_04435_gb300 import vlb
    n, wall = (48, 48, 48), (0, 0, 0)
    xyz, nxt = jittered_tangle(n, wall, 25, seed, jitter, spacing)
    g, r = pair(tparams(n, wall), xyz, nxt)
    for _ in range(3):
        g.run_phases(vlb.PHASE_REMESH)
        r.run_phases(oracle.PHASE_REMESH)
        assert_same_points(g, r)


def test_remesh_walls_bit_exact():
    import oracle
    from paper_2108_04435_gb300 import vlb
    n, wall = (40, 36, 44), (1, 1, 1)
    xyz, nxt = jittered_tangle(n, wall, 20, 7, 0.25, 0.9)
    g, r = pair(tparams(n, wall), xyz, nxt)
    g.run_phases(vlb.PHASE_REMESH)
    r.run_phases(oracle.PHASE_REMESH)
    assert_same_points(g, r)


def test_reconnect_squares_hand_case():
    import oracle
    from paper_2108_04435_gb300 import vlb
    sq = np.array([(0, 0), (0.8, 0), (1.6, 0), (1.6, 0.8), (1.6, 1.6), (0.8, 1.6), (0, 1.6), (0, 0.8)])
    A = np.c_[sq + [2.0, 3.0], np.full(8, 4.0)]
    B = np.c_[sq + [2.0 + 1.6 + 0.5, 3.0], np.full(8, 4.0)]
    xyz = np.r_[A, B]
    nxt = np.r_[(np.arange(8) + 1) % 8, 8 + (np.arange(8) + 1) % 8].astype(np.int32)
    g, r = pair(tparams((8, 8, 8), (0, 0, 0)), xyz, nxt)
    g.run_phases(vlb.PHASE_RECONNECT)
    r.run_phases(oracle.PHASE_RECONNECT)
    assert_same_points(g, r)
    assert g.stats()[7] == 1


@pytest.mark.parametrize("seed,wall", [(0, (0, 0, 0)), (1, (0, 0, 0)), (2, (1, 1, 1)), (3, (0, 1, 0))])
def test_reconnect_dense_tangle_bit_exact(seed, wall):
    """Dense jittered tangle: many mutual-nearest pairs and conflicting exchanges."""
    import oracle
    from paper_2108_04435_gb300 import vlb
    n = (24, 24, 24)
    xyz, nxt = jittered_tangle(n, wall, 40, seed, 0.3, 0.8)
    g, r = pair(tparams(n, wall), xyz, nxt)
    for _ in range(2):
        g.run_phases(vlb.PHASE_RECONNECT)
        r.run_phases(oracle.PHASE_RECONNECT)
        assert_same_points(g, r)
    assert r.stats()[7] > 0


@pytest.mark.parametrize("rel", [-1e-12, 1e-12])
def test_reconnect_at_the_threshold_far_from_origin(rel):
    """Two squares whose facing sides are dxi_max (1 + rel) apart, 250 cells
    along a 256-cell axis: the pairs just inside dxi_max reconnect and those
    just outside do not, exactly as the FP64 oracle decides (the FP32 bound
    that prunes the nearest-point search drops no point inside dxi_max)."""
    import oracle
    from paper_2108_04435_gb300 import vlb
    p = tparams((256, 8, 8), (0, 0, 0))
    d = p["dxi_max"] * (1.0 + rel)
    sq = 1.2 * np.array([(0, 0), (1, 0), (2, 0), (2, 1), (2, 2), (1, 2), (0, 2), (0, 1)])
    A = np.c_[sq + [250.0, 2.0], np.full(8, 4.0)]
    B = np.c_[sq + [252.4 + d, 2.0], np.full(8, 4.0)]
    xyz = np.r_[A, B]
    nxt = np.r_[(np.arange(8) + 1) % 8, 8 + (np.arange(8) + 1) % 8].astype(np.int32)
    g, r = pair(p, xyz, nxt)
    g.run_phases(vlb.PHASE_RECONNECT)
    r.run_phases(oracle.PHASE_RECONNECT)
    assert_same_points(g, r)
    assert r.stats()[7] == (1 if rel < 0 else 0)


def test_remesh_then_reconnect_past_the_grid_span():
    """Remeshing doubles the points within one launch sequence, so the
    reconnection kernels, whose grids cover the count known before it (rounded
    up to a power of two), stride over the points beyond their grid."""
    import oracle
    from paper_2108_04435_gb300 import vlb
    n, wall = (24, 24, 24), (0, 0, 0)
    xyz, nxt = jittered_tangle(n, wall, 20, 5, 0.02, 1.02)
    assert 512 < len(xyz) < 1024
    g, r = pair(tparams(n, wall), xyz, nxt)
    g.run_phases(vlb.PHASE_REMESH | vlb.PHASE_RECONNECT)
    r.run_phases(oracle.PHASE_REMESH | oracle.PHASE_RECONNECT)
    assert_same_points(g, r)
    assert r.n_points() > 1024 and r.stats()[7] > 0


def test_empty_and_capacity():
    from paper_2108_04435_gb300 import inputs, vlb
    p = tparams((16, 16, 16), (0, 0, 0), max_points=100)
    g = vlb.Channel(p)
    g.step(2)  # no filaments
    assert g.n_points() == 0
    xyz, nxt = inputs.ring((8, 8, 8), (0, 0, 1), 4.0, npts=150)
    with pytest.raises(vlb.VlbError) as e:
        g.seed(xyz, nxt)
    assert e.value.code == -3
    bad = np.array([1, 1, 2], np.int32)
    with pytest.raises(vlb.VlbError) as e:
        g.seed(xyz[:3], bad)
    assert e.value.code == -4
    # splits beyond max_points are reported, not written
    xyz, nxt = inputs.ring((8, 8, 8), (0, 0, 1), 7.0, npts=60)  # chord 0.73 -> no split
    p2 = tparams((16, 16, 16), (0, 0, 0), max_points=70)
    g2 = vlb.Channel(p2)
    xyz2, nxt2 = inputs.ring((8, 8, 8), (0, 0, 1), 7.0, npts=40)  # chord 1.1 > dxi_max
    g2.seed(xyz2, nxt2)
    rc = g2.run_phases(vlb.PHASE_REMESH, raise_on_error=False)
    assert rc == -3
    assert g2.n_points() == 40


@pytest.mark.parametrize("phase", ["remesh", "reconnect", "step"])
def test_seeded_small_loop_deleted(phase):
    """A seeded loop of four points dies in the first remesh or reconnection
    pass that follows the seeding, even when that pass removes, exchanges and
    cuts nothing: the finishers skip the small-component check only when
    nothing could have shortened a loop, and seeding asks for one check."""
    import oracle
    from paper_2108_04435_gb300 import inputs, vlb
    n, wall = (32, 32, 32), (0, 0, 0)
    big, nbig = inputs.ring((16.0, 16.0, 8.0), (0.0, 0.0, 1.0), 6.0, npts=48)
    small, nsmall = inputs.ring((16.0, 16.0, 24.0), (0.0, 0.0, 1.0), 0.45, npts=4)
    xyz, nxt = inputs.concat([(big, nbig), (small, nsmall)])
    p = tparams(n, wall, dxi_min=0.2, dxi_max=0.95)
    g, r = pair(p, xyz, nxt)
    if phase == "remesh":
        g.run_phases(vlb.PHASE_REMESH)
        r.run_phases(oracle.PHASE_REMESH)
    elif phase == "reconnect":
        g.run_phases(vlb.PHASE_RECONNECT)
        r.run_phases(oracle.PHASE_RECONNECT)
    else:  # a whole step: the advance is FP32 against FP64, the topology still exact
        g.step(1)
        r.step(1)
        assert g.n_points() == r.n_points() == len(nbig)
        assert np.array_equal(g.read(vlb.FIELD_NEXT), r.read(oracle.FIELD_NEXT))
        pg, pr = g.read(vlb.FIELD_POS), r.read(oracle.FIELD_POS)
        assert np.linalg.norm(pg - pr) < 1e-5 * np.linalg.norm(pr)
        return
    assert_same_points(g, r)
    assert g.n_points() == len(nbig)
