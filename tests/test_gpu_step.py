"""Whole coupled step through the C ABI vs the oracle, at the sizes the
benchmark uses, plus multi-step drift and the smoke entry point."""
import numpy as np
import pytest

from gpu_util import pair, rel_l2

pytestmark = pytest.mark.gpu


def compare_step(g, r, xyz, n, wall, tol=1e-5, line_tol=1e-9):
    import oracle
    from paper_2108_04435_gb300 import vlb
    f_g = g.read(vlb.FIELD_FSTAR)
    f_r = r.read(oracle.FIELD_FSTAR)
    c, w, _ = oracle.lattice()
    rest = (w * r.params["rho0"])[:, None]
    assert rel_l2(f_g, f_r) < tol
    assert rel_l2(g.read(vlb.FIELD_FDEV), f_r - rest) < tol
    assert rel_l2(g.read(vlb.FIELD_U), r.read(oracle.FIELD_U)) < tol
    assert rel_l2(g.read(vlb.FIELD_FORCE), r.read(oracle.FIELD_FORCE)) < tol
    assert np.array_equal(g.read(vlb.FIELD_NEXT), r.read(oracle.FIELD_NEXT))
    pg, pr = g.read(vlb.FIELD_POS), r.read(oracle.FIELD_POS)
    assert rel_l2(g.read(vlb.FIELD_VEL), r.read(oracle.FIELD_VEL)) < tol
    assert abs(g.line_length() / r.line_length() - 1) < line_tol
    prof_g, prof_r = g.read(vlb.FIELD_LINE_PROFILE), r.read(oracle.FIELD_LINE_PROFILE)
    assert np.abs(prof_g - prof_r).sum() < max(line_tol, 1e-9) * prof_r.sum()
    return pg, pr


def test_ring32_one_step():
    from paper_2108_04435_gb300 import configs
    p, xyz, nxt = configs.config("ring32")
    g, r = pair(p, xyz, nxt)
    g.step(1)
    r.step(1)
    pg, pr = compare_step(g, r, xyz, p["n"], p["wall"])
    assert rel_l2(pg - xyz, pr - xyz) < 1e-5


def test_ring32_twenty_steps():
    from paper_2108_04435_gb300 import configs
    p, xyz, nxt = configs.config("ring32")
    g, r = pair(p, xyz, nxt)
    g.step(20)
    r.step(20)
    pg, pr = compare_step(g, r, xyz, p["n"], p["wall"], tol=2e-5, line_tol=1e-7)
    d = pg - pr
    assert np.abs(d).max() < 1e-6


def test_channel_64x64x256_one_step():
    """The benchmark workload: closed channel, heater, 20 rings (~1.2k points)."""
    from paper_2108_04435_gb300 import configs
    p, xyz, nxt = configs.config("channel64x64x256")
    g, r = pair(p, xyz, nxt)
    g.step(1)
    r.step(1)
    pg, pr = compare_step(g, r, xyz, p["n"], p["wall"])
    assert rel_l2(pg - xyz, pr - xyz) < 1e-5


def test_runs_are_bitwise_reproducible():
    """Two runs of the benchmark workload from the same seed give identical
    populations, force grid and points after 30 steps."""
    from paper_2108_04435_gb300 import configs, vlb
    p, xyz, nxt = configs.config("channel64x64x256")
    out = []
    for _ in range(2):
        g = vlb.Channel(p)
        g.seed(xyz, nxt)
        g.step(30)
        out.append([g.read(w) for w in (vlb.FIELD_FSTAR, vlb.FIELD_FORCE, vlb.FIELD_POS, vlb.FIELD_NEXT)])
        g.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_smoke_entry():
    import __graft_entry__
    __graft_entry__.smoke()


@pytest.mark.parametrize("name,steps,fused", [("channel64x64x256", 20, "0"), ("channel64x64x256_lines", 20, "0"),
                                              ("box128", 12, "0"), ("box128", 12, "1")])
def test_overlapped_graph_steps_match_sequential(name, steps, fused, monkeypatch):
    """The 8-step graphs run the lattice pass of each step alongside the
    remesh and reconnection of the step before, on a second stream; with the
    overlap off the same graphs keep every step in sequence.  Populations,
    force grid, points, links and statistics agree bit for bit (walls with
    open lines; the periodic box at 16.9k points, with fixed-point split sums
    and, forced by VLB_FUSED_EOM=1, with the Biot-Savart kernel applying the
    equation of motion)."""
    from paper_2108_04435_gb300 import configs, vlb
    monkeypatch.setenv("VLB_FUSED_EOM", fused)
    p, xyz, nxt = configs.config(name)
    out = []
    for overlap in (True, False):
        g = vlb.Channel(p)
        g.set_overlap(overlap)
        g.seed(xyz, nxt)
        g.step(steps)
        out.append([g.read(w) for w in (vlb.FIELD_FSTAR, vlb.FIELD_FORCE, vlb.FIELD_POS, vlb.FIELD_NEXT,
                                         vlb.FIELD_STATS)])
        g.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_overlap_switch_mid_run():
    """Turning the overlap off and on between steps recaptures the 8-step
    graphs and continues the same trajectory as a run that never switched."""
    from paper_2108_04435_gb300 import configs, vlb
    p, xyz, nxt = configs.config("channel64x64x256")
    out = []
    for switch in (False, True):
        g = vlb.Channel(p)
        g.seed(xyz, nxt)
        g.step(8)
        if switch:
            g.set_overlap(False)
        g.step(8)
        if switch:
            g.set_overlap(True)
        g.step(8)
        out.append([g.read(w) for w in (vlb.FIELD_FSTAR, vlb.FIELD_POS, vlb.FIELD_NEXT)])
        g.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", [0, 1], ids=["f32", "f16"])
def test_cache_hints_change_nothing(storage, monkeypatch):
    """The evict-first hints on the population traffic (on by default when a
    population buffer fits in L2) change where lines live, not a single
    value: 16 coupled steps agree bit for bit with the hints forced off."""
    from paper_2108_04435_gb300 import configs, vlb
    p, xyz, nxt = configs.config("channel64x64x256")
    p["storage"] = storage
    out = []
    for hint in ("1", "0"):
        monkeypatch.setenv("VLB_LBM_STREAM_HINT", hint)
        g = vlb.Channel(p)
        g.seed(xyz, nxt)
        g.step(16)
        out.append([g.read(w) for w in (vlb.FIELD_FSTAR, vlb.FIELD_FORCE, vlb.FIELD_POS, vlb.FIELD_NEXT)])
        g.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_line_length_after_step_is_current():
    """vlb_step leaves the line length of the new points with the status; it
    equals a fresh computation after the same steps, and a call that changes
    nothing (an empty phase mask) makes the next read compute it again."""
    from paper_2108_04435_gb300 import configs, vlb
    p, xyz, nxt = configs.config("channel64x64x256")
    g = vlb.Channel(p)
    g.seed(xyz, nxt)
    l0 = g.line_length()
    g.step(5)
    cached = g.line_length()
    g.run_phases(0)
    fresh = g.line_length()
    g.close()
    assert cached == fresh and cached != l0


def test_async_calls_in_flight_match_blocking_steps():
    """Several vlb_step_async calls in flight, each completed in order by
    vlb_query.  One-step calls run split over two streams (the remesh and
    reconnection of one call beside the lattice pass of the next); every
    call's own status (points, mass, line length, max Mach, step count)
    equals that of a blocking vlb_step(1) channel after the same steps, and
    the final points, populations and status are identical.  The queue holds
    VLB_ASYNC_DEPTH calls; vlb_step refuses while calls are queued."""
    import torch
    from paper_2108_04435_gb300 import configs, vlb
    p, xyz, nxt = configs.config("channel64x64x256")
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    a = vlb.Channel(p, stream=sa)
    b = vlb.Channel(p, stream=sb)
    a.seed(xyz, nxt)
    b.seed(xyz, nxt)
    ref = []
    for _ in range(6):
        b.step(1)
        ref.append(b.stats())
    got = []
    for k in range(6):
        a.step_async(1)
        if k >= 2:  # three calls in flight, then one completed per call
            while not a.query():
                pass
            got.append(a.query_stats())
    while len(got) < 6:
        while not a.query():
            pass
        got.append(a.query_stats())
    for r, g in zip(ref, got):  # points, mass, line length, max Mach, steps
        assert all(g[k] == r[k] for k in (0, 2, 3, 4, 9)), (g[:10], r[:10])
    assert np.array_equal(a.read(vlb.FIELD_POS), b.read(vlb.FIELD_POS))
    assert np.array_equal(a.read(vlb.FIELD_FSTAR), b.read(vlb.FIELD_FSTAR))
    assert np.array_equal(a.stats()[:5], b.stats()[:5])
    for _ in range(vlb.ASYNC_DEPTH):
        a.step_async(1)
    with pytest.raises(vlb.VlbError):
        a.step_async(1)
    with pytest.raises(vlb.VlbError):
        a.step(1)
    for _ in range(vlb.ASYNC_DEPTH):
        while not a.query():
            pass
    a.step(1)
    a.close()
    b.close()
