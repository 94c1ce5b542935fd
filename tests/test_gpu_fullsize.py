"""Parity with the oracle at the sizes that are benchmarked.

- The 128 x 128 x 1024 closed channel (16.8M cells, 1000 seeded rings of
  ~86k points) for one lattice pass and one filament advance: the stage-1
  velocity, the displacement, the spread force grid and the velocity field
  at relative L2 1e-5.  This runs the spatially ordered Biot-Savart sum at its
  natural size (several hundred source groups per split, origins up to 1024
  cells from zero) and the equation of motion applied inside it, with the
  lattice on the benchmark's grid.  The lattice uses FP32 storage here; the
  FP16/BF16 formats have their own bounds below.
- Remeshing and reconnection from identical inputs of more than 20k points,
  bit for bit: the single-block compactions then work through many chunks of
  1024 points.
- One lattice pass of 128^3 with FP16 and BF16 storage within the bounds the
  reduced formats are stated to keep, periodic and with walls on every axis
  (where most blocks take the two-cell body without the wall logic).
- One whole coupled step of the 128^3 periodic counterflow box (~18.5k points).
"""
import numpy as np
import pytest

from gpu_util import pair, rel_l2, same_lattice_state

pytestmark = pytest.mark.gpu


def unwrap(d, n, wall):
    L = np.array(n, float)
    for a in range(3):
        if not wall[a]:
            d[:, a] -= L[a] * np.round(d[:, a] / L[a])
    return d


def test_largest_channel_advance_parity():
    import oracle
    from paper_2108_04435_gb300 import configs, vlb
    p, xyz, nxt = configs.config("channel128x128x1024")
    p["storage"] = 0
    assert len(nxt) > 80000
    g, r = pair(p, xyz, nxt)
    same_lattice_state(g, r, seed=41, amp=2e-3)
    g.run_phases(vlb.PHASE_LBM | vlb.PHASE_VFM)
    r.run_phases(oracle.PHASE_LBM | oracle.PHASE_VFM)
    e_u = rel_l2(g.read(vlb.FIELD_U), r.read(oracle.FIELD_U))
    e_v = rel_l2(g.read(vlb.FIELD_VEL), r.read(oracle.FIELD_VEL))
    x0 = np.asarray(xyz)
    dg = unwrap(g.read(vlb.FIELD_POS) - x0, p["n"], p["wall"])
    dr = unwrap(r.read(oracle.FIELD_POS) - x0, p["n"], p["wall"])
    e_d = rel_l2(dg, dr)
    print("benchmark channel: velocity field", e_u, "point velocity", e_v, "displacement", e_d)
    assert e_u < 1e-5 and e_v < 1e-5 and e_d < 1e-5
    assert rel_l2(g.read(vlb.FIELD_FORCE), r.read(oracle.FIELD_FORCE)) < 1e-5
    # Eq. 18 per plane and the mass: FP64 sums of warp partials of the FP32
    # density and velocity deviations
    assert rel_l2(g.read(vlb.FIELD_PLANE_VS), r.read(oracle.FIELD_PLANE_VS)) < 1e-5
    m_g, m_r = g.stats()[2], r.stats()[2]
    print("mass", m_g, m_r, abs(m_g / m_r - 1))
    assert abs(m_g / m_r - 1) < 1e-9
    g.close()
    r.close()


def test_topology_bit_exact_above_20k_points():
    import oracle
    from paper_2108_04435_gb300 import configs, inputs, vlb
    n, wall = (128, 128, 128), (0, 0, 0)
    xyz, nxt = inputs.random_rings(n, wall, 400, 2.0, 12.0, 17, spacing=0.8, min_sep=0.0)
    rng = np.random.default_rng(117)
    xyz = np.mod(xyz + 0.3 * rng.uniform(-1, 1, xyz.shape), 128.0)
    assert len(nxt) > 20000
    p = configs.base_params(n, wall, 1.9, couple=0, max_points=65536)
    g, r = pair(p, xyz, nxt)
    for _ in range(2):
        g.run_phases(vlb.PHASE_REMESH | vlb.PHASE_RECONNECT)
        r.run_phases(oracle.PHASE_REMESH | oracle.PHASE_RECONNECT)
        assert g.n_points() == r.n_points()
        assert np.array_equal(g.read(vlb.FIELD_NEXT), r.read(oracle.FIELD_NEXT))
        assert np.array_equal(g.read(vlb.FIELD_POS), r.read(oracle.FIELD_POS))
        assert np.array_equal(g.stats()[5:9], r.stats()[5:9])
    s = r.stats()
    assert s[5] > 0 and s[6] > 0 and s[7] > 0  # splits, merges and exchanges all happened


@pytest.mark.parametrize("walls", [(0, 0, 0), (1, 1, 1)], ids=["periodic", "walls"])
@pytest.mark.parametrize("storage,bound", [(1, 1e-3), (2, 8e-3)], ids=["f16", "bf16"])
def test_reduced_storage_pass_128(storage, bound, walls):
    import oracle
    from paper_2108_04435_gb300 import configs, vlb
    c, w, _ = oracle.lattice()
    p = configs.base_params((128, 128, 128), walls, 1.9, couple=0, max_points=8, storage=storage,
                            heater_vn=0.01 if walls[2] else 0.0, init_vn=[0.003, -0.002, 0.01])
    g, r = pair(p)
    same_lattice_state(g, r, seed=43, amp=1e-2, force_amp=2e-4)
    g.run_phases(vlb.PHASE_LBM)
    r.run_phases(oracle.PHASE_LBM)
    f_r = r.read(oracle.FIELD_FSTAR)
    e_dev = rel_l2(g.read(vlb.FIELD_FDEV), f_r - (w * p["rho0"])[:, None])
    e_u = rel_l2(g.read(vlb.FIELD_U), r.read(oracle.FIELD_U))
    print("storage", storage, "deviation", e_dev, "velocity", e_u)
    assert e_dev < bound and e_u < bound


def test_box128_whole_step():
    import oracle
    from paper_2108_04435_gb300 import configs, vlb
    p, xyz, nxt = configs.config("box128")
    g, r = pair(p, xyz, nxt)
    g.step(1)
    r.step(1)
    c, w, _ = oracle.lattice()
    f_r = r.read(oracle.FIELD_FSTAR)
    assert rel_l2(g.read(vlb.FIELD_FDEV), f_r - (w * p["rho0"])[:, None]) < 1e-5
    assert rel_l2(g.read(vlb.FIELD_FORCE), r.read(oracle.FIELD_FORCE)) < 1e-5
    assert rel_l2(g.read(vlb.FIELD_VEL), r.read(oracle.FIELD_VEL)) < 1e-5
    assert np.array_equal(g.read(vlb.FIELD_NEXT), r.read(oracle.FIELD_NEXT))
    x0 = np.asarray(xyz)
    dg = unwrap(g.read(vlb.FIELD_POS) - x0, p["n"], p["wall"])
    dr = unwrap(r.read(oracle.FIELD_POS) - x0, p["n"], p["wall"])
    assert rel_l2(dg, dr) < 1e-5
    assert abs(g.line_length() / r.line_length() - 1) < 1e-9
