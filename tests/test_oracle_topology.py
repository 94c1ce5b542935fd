"""Pins of the oracle's remeshing and reconnection (Sec. II.A; Sec. III.B).

The paper fixes the resolution [dxi_min, dxi_max] = [0.70, 0.95] (Sec. III)
and that legs are exchanged when two vortices come within the resolution;
the rules that realise this are readings (listed in the oracle's header).
These tests pin them with hand-worked cases and invariants:
- two antiparallel square loops 0.5 apart reconnect into one loop, with the
  exchange worked out by hand below; co-directional loops never reconnect; an
  isolated ring never reconnects;
- a regular ring whose segments all exceed dxi_max gets one arc-midpoint
  per segment, on the circle to O(l^4);
- a ring of over-fine segments coarsens without moving points, never removes
  two neighbours in one pass, and stops once no merge keeps the merged
  segment within dxi_max;
- loops of fewer than five points are deleted.
"""
import numpy as np
import pytest

from paper_2108_04435_gb300 import configs, inputs


def tparams(n=(8, 8, 8), wall=(0, 0, 0), **kw):
    kw.setdefault("couple", 0)
    kw.setdefault("max_points", 1024)
    return configs.base_params(n, wall, 1.9, **kw)


SQUARE = np.array([(0, 0), (0.8, 0), (1.6, 0), (1.6, 0.8), (1.6, 1.6), (0.8, 1.6), (0, 1.6), (0, 0.8)])


def two_squares(gap=0.5, reverse_b=False):
    A = np.c_[SQUARE + [2.0, 3.0], np.full(8, 4.0)]
    B = np.c_[SQUARE + [2.0 + 1.6 + gap, 3.0], np.full(8, 4.0)]
    na = (np.arange(8) + 1) % 8
    nb = (np.arange(8) + 1) % 8
    if reverse_b:
        nb = (np.arange(8) - 1) % 8
    return np.r_[A, B], np.r_[na, 8 + nb].astype(np.int32)


def loops_of(nxt):
    seen = np.zeros(len(nxt), bool)
    sizes = []
    for s in range(len(nxt)):
        if seen[s]:
            continue
        k, j = 0, s
        while not seen[j]:
            seen[j] = True
            j = nxt[j]
            k += 1
        sizes.append(k)
    return sorted(sizes)


def test_antiparallel_squares_reconnect_as_worked_by_hand(oracle_mod):
    """A's right side runs up (a2 -> a3 -> a4) and B's left side runs down
    (b6 -> b7 -> b0), 0.5 apart.  Mutual nearest pairs: (a2,b0), (a3,b7),
    (a4,b6), all at d = 0.5.  For (a2,b0) the best exchange is on segments
    a2->a3 and b7->b0 (new links a2->b0 and b7->a3, length 1.0 instead of 1.6);
    it is applied first (smallest i) and claims a2, a3, b7, b0, which blocks
    the exchanges proposed for the other two pairs (both use a3)."""
    xyz, nxt = two_squares()
    ch = oracle_mod.Channel(tparams())
    ch.seed(xyz, nxt)
    ch.run_phases(oracle_mod.PHASE_RECONNECT)
    expect = np.r_[(np.arange(8) + 1) % 8, 8 + (np.arange(8) + 1) % 8]
    expect[2] = 8      # a2 -> b0
    expect[15] = 3     # b7 -> a3
    assert np.array_equal(ch.read(oracle_mod.FIELD_NEXT), expect)
    assert ch.stats()[7] == 1
    assert loops_of(ch.read(oracle_mod.FIELD_NEXT)) == [16]


def test_parallel_squares_do_not_reconnect(oracle_mod):
    xyz, nxt = two_squares(reverse_b=True)
    ch = oracle_mod.Channel(tparams())
    ch.seed(xyz, nxt)
    ch.run_phases(oracle_mod.PHASE_RECONNECT)
    assert np.array_equal(ch.read(oracle_mod.FIELD_NEXT), nxt)
    assert ch.stats()[7] == 0


def test_squares_out_of_range_do_not_reconnect(oracle_mod):
    xyz, nxt = two_squares(gap=0.96)
    ch = oracle_mod.Channel(tparams())
    ch.seed(xyz, nxt)
    ch.run_phases(oracle_mod.PHASE_RECONNECT)
    assert ch.stats()[7] == 0


def test_isolated_rings_never_reconnect(oracle_mod):
    p = tparams(n=(64, 64, 64))
    xyz, nxt = inputs.concat([inputs.ring((20, 32, 32), (0, 0, 1), 8.0), inputs.ring((44, 32, 32), (0, 1, 0), 6.0)])
    ch = oracle_mod.Channel(p)
    ch.seed(xyz, nxt)
    for _ in range(3):
        ch.run_phases(oracle_mod.PHASE_RECONNECT)
    assert ch.stats()[7] == 0
    assert np.array_equal(ch.read(oracle_mod.FIELD_NEXT), nxt)


def test_split_regular_ring(oracle_mod):
    N, R = 48, 8.0   # chord 2R sin(pi/N) = 1.047 > dxi_max
    c = np.array([16.0, 16.0, 16.0])
    xyz, nxt = inputs.ring(c, (0, 0, 1), R, npts=N)
    ch = oracle_mod.Channel(tparams(n=(32, 32, 32)))
    ch.seed(xyz, nxt)
    ch.run_phases(oracle_mod.PHASE_REMESH)
    pos, nn = ch.read(oracle_mod.FIELD_POS), ch.read(oracle_mod.FIELD_NEXT)
    assert len(nn) == 2 * N
    assert np.array_equal(nn[:N], N + np.arange(N))
    assert np.array_equal(nn[N:], (np.arange(N) + 1) % N)
    assert np.array_equal(pos[:N], xyz)
    # arc midpoint: on the circle to O(l^4/R^3), half-way in angle
    assert np.abs(np.linalg.norm(pos[N:] - c, axis=1) - R).max() < 1e-4
    ang = np.arctan2(pos[N:, 1] - c[1], pos[N:, 0] - c[0])
    want = np.arctan2(xyz[:, 1] - c[1], xyz[:, 0] - c[0]) + np.pi / N
    assert np.abs(np.angle(np.exp(1j * (ang - want)))).max() < 1e-12
    assert ch.stats()[5] == N


def test_merge_fine_ring_invariants(oracle_mod):
    N, R = 128, 8.0  # chord 0.393 < dxi_min, two chords 0.785 <= dxi_max
    xyz, nxt = inputs.ring((16, 16, 16), (0, 0, 1), R, npts=N)
    p = tparams(n=(32, 32, 32))
    ch = oracle_mod.Channel(p)
    ch.seed(xyz, nxt)
    prev_n, passes = N, 0
    while True:
        ch.run_phases(oracle_mod.PHASE_REMESH)
        pos, nn = ch.read(oracle_mod.FIELD_POS), ch.read(oracle_mod.FIELD_NEXT)
        # survivors are original points, kept in the original cyclic order
        idx = [int(np.argmin(np.linalg.norm(xyz - q, axis=1))) for q in pos]
        assert np.abs(pos - xyz[idx]).max() == 0.0
        orig = np.array(idx)
        if passes == 0:
            gone = sorted(set(range(N)) - set(idx))
            assert all((g + 1) % N not in gone for g in gone)   # no two neighbours removed
        assert np.array_equal(orig[nn], np.sort(orig)[(np.searchsorted(np.sort(orig), orig) + 1) % len(orig)])
        passes += 1
        if len(nn) == prev_n:
            break
        prev_n = len(nn)
        assert passes < 20
    l = np.linalg.norm(pos[nn] - pos, axis=1)
    assert l.max() <= p["dxi_max"]
    # no merge candidate remains
    prv = np.empty_like(nn)
    prv[nn] = np.arange(len(nn))
    for i in range(len(nn)):
        short = min(l[prv[i]], l[i]) < p["dxi_min"]
        assert not (short and np.linalg.norm(pos[nn[i]] - pos[prv[i]]) <= p["dxi_max"])


def test_small_loops_deleted(oracle_mod):
    p = tparams(n=(16, 16, 16))
    ring4 = inputs.ring((4, 4, 4), (0, 0, 1), 0.6, npts=4)      # side 0.85
    ring5 = inputs.ring((10, 10, 10), (0, 0, 1), 0.68, npts=5)  # side 0.80
    xyz, nxt = inputs.concat([ring4, ring5])
    ch = oracle_mod.Channel(p)
    ch.seed(xyz, nxt)
    ch.run_phases(oracle_mod.PHASE_REMESH)
    assert ch.n_points() == 5
    assert np.array_equal(ch.read(oracle_mod.FIELD_POS), xyz[4:])
    assert ch.stats()[8] == 4


@pytest.mark.parametrize("seed", [0, 1])
def test_tangle_topology_invariants(oracle_mod, seed):
    """A seeded tangle stepped with remesh + reconnect keeps next/prev a
    permutation of closed loops of at least five points."""
    p = tparams(n=(32, 32, 32), couple=1, init_vn=[0.0, 0.0, 0.0116])
    xyz, nxt = inputs.random_rings((32, 32, 32), (0, 0, 0), 12, 3.0, 6.0, seed)
    ch = oracle_mod.Channel(p)
    ch.seed(xyz, nxt)
    ch.step(30)
    nn = ch.read(oracle_mod.FIELD_NEXT)
    assert np.array_equal(np.sort(nn), np.arange(len(nn)))
    assert min(loops_of(nn)) >= 5
    pos = ch.read(oracle_mod.FIELD_POS)
    d = pos[nn] - pos
    d -= 32 * np.round(d / 32)
    assert np.linalg.norm(d, axis=1).max() <= p["dxi_max"] + 0.1


@pytest.mark.parametrize("rel,split", [(-1e-9, False), (1e-9, True)])
def test_split_threshold_is_dxi_max(oracle_mod, rel, split):
    # Sec. III's upper spacing 0.95: a regular 64-gon whose chord lies just
    # below it is left alone, just above it every segment is split
    N = 64
    R = 0.95 * (1 + rel) / (2 * np.sin(np.pi / N))
    xyz, nxt = inputs.ring((16.0, 16.0, 16.0), (0, 0, 1), R, npts=N)
    ch = oracle_mod.Channel(tparams(n=(32, 32, 32)))
    ch.seed(xyz, nxt)
    ch.run_phases(oracle_mod.PHASE_REMESH)
    assert ch.n_points() == (2 * N if split else N)


@pytest.mark.parametrize("rel,removed", [(-1e-9, True), (1e-9, False)])
def test_removal_threshold_is_dxi_min(oracle_mod, rel, removed):
    # Sec. III's lower spacing 0.70 on a sharp kink, where it is the binding
    # condition: a tip point at distance L from both of its neighbours, which
    # sit 0.8 apart on a regular ring (so the merged segment stays within
    # 0.95).  L just below 0.70 removes the tip and nothing else; just above,
    # the loop is unchanged.
    N, chord = 40, 0.8
    R = chord / (2 * np.sin(np.pi / N))
    c = np.array([32.0, 32.0, 32.0])
    th = 2 * np.pi * np.arange(N) / N
    ring = np.stack([c[0] + R * np.cos(th), c[1] + R * np.sin(th), np.full(N, c[2])], axis=1)
    mid = 0.5 * (ring[0] + ring[1])
    out = (mid - c) / np.linalg.norm(mid - c)
    L = 0.70 * (1 + rel)
    tip = mid + np.sqrt(L * L - (chord / 2) ** 2) * out
    xyz = np.concatenate([ring[:1], tip[None], ring[1:]])
    nxt = (np.arange(N + 1) + 1) % (N + 1)
    ch = oracle_mod.Channel(tparams(n=(64, 64, 64)))
    ch.seed(xyz, nxt)
    ch.run_phases(oracle_mod.PHASE_REMESH)
    pos = ch.read(oracle_mod.FIELD_POS)
    want = np.delete(xyz, 1, axis=0) if removed else xyz
    assert np.array_equal(pos, want)
    assert np.array_equal(ch.read(oracle_mod.FIELD_NEXT), (np.arange(len(want)) + 1) % len(want))
