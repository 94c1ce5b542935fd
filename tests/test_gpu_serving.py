"""Serving on the GPU: runs admitted together overlap on separate streams and
each gives the same result as when it is served alone, bit for bit (every
reduction of the step has a fixed order and the force spreading accumulates
in fixed point, so the interleaving of runs on the device cannot change a
result)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def small_requests():
    from paper_2108_04435_gb300 import configs
    reqs = configs.serving_requests(5, 50.0, 7, 60, grids=((32, 32, 32), (48, 48, 48), (64, 64, 64)),
                                    points=(100, 800))
    for r in reqs:
        n = r["params"]["n"]
        r["cells"] = n[0] * n[1] * n[2]
    return reqs


def fields():
    from paper_2108_04435_gb300 import vlb
    return (vlb.FIELD_FSTAR, vlb.FIELD_FORCE, vlb.FIELD_POS, vlb.FIELD_NEXT, vlb.FIELD_STATS)


def test_same_alone_and_in_the_mix():
    """Populations, force grid, points, links and the status record of every
    run are identical, bit for bit, served alone and served in the mix."""
    import copy
    from paper_2108_04435_gb300 import serve, vlb
    reqs = small_requests()
    budget = sum(vlb.channel_bytes(r["params"]) for r in reqs)
    mix, summary = serve.serve_gpu(copy.deepcopy(reqs), budget_bytes=budget, max_slots=5, slice_steps=20,
                                   realtime=False, snapshot=fields())
    assert summary["failed"] == 0 and summary["peak_slots"] >= 2
    for r in reqs:
        alone, _ = serve.serve_gpu([copy.deepcopy(r)], budget_bytes=budget, max_slots=1, slice_steps=20,
                                   realtime=False, snapshot=fields())
        a, m = alone[0], mix[r["id"]]
        assert a.steps == m.steps == 60
        assert a.n_points == m.n_points
        assert a.line_length == m.line_length
        for w in fields():
            if w == vlb.FIELD_STATS:  # all but the device bytes, which follow the capacity
                assert np.array_equal(np.delete(a.state[w], 10), np.delete(m.state[w], 10))
            else:
                assert np.array_equal(a.state[w], m.state[w]), w


def test_served_request_matches_the_oracle():
    """A request served in a mix of three ends where the FP64 oracle ends
    after the same steps, within the whole-step tolerance."""
    import copy

    import oracle
    from gpu_util import rel_l2
    from paper_2108_04435_gb300 import configs, serve, vlb
    reqs = configs.serving_requests(3, 50.0, 21, 20, grids=((32, 32, 32), (40, 40, 40)), points=(100, 300))
    budget = sum(vlb.channel_bytes(r["params"]) for r in reqs)
    res, summary = serve.serve_gpu(copy.deepcopy(reqs), budget_bytes=budget, max_slots=3, slice_steps=10,
                                   realtime=False, snapshot=fields())
    assert summary["failed"] == 0 and summary["peak_slots"] >= 2
    req = reqs[0]
    r = oracle.Channel(req["params"])
    r.seed(req["xyz"], req["next"])
    r.step(req["steps"])
    st = res[0].state
    c, w, _ = oracle.lattice()
    f_r = r.read(oracle.FIELD_FSTAR)
    rest = (w * req["params"]["rho0"])[:, None]
    assert rel_l2(st[vlb.FIELD_FSTAR] - rest, f_r - rest) < 2e-5
    assert np.array_equal(st[vlb.FIELD_NEXT], r.read(oracle.FIELD_NEXT))
    x0 = np.asarray(req["xyz"])
    n = np.array(req["params"]["n"], float)
    dg, dr = st[vlb.FIELD_POS] - x0, r.read(oracle.FIELD_POS) - x0
    for d in (dg, dr):
        d -= n * np.round(d / n)
    assert rel_l2(dg, dr) < 2e-5


def test_budget_limits_concurrency():
    import copy
    from paper_2108_04435_gb300 import serve, vlb
    reqs = small_requests()
    biggest = max(vlb.channel_bytes(r["params"]) for r in reqs)
    res, summary = serve.serve_gpu(copy.deepcopy(reqs), budget_bytes=biggest, max_slots=5, slice_steps=20,
                                   realtime=False)
    assert summary["failed"] == 0
    assert summary["peak_bytes"] <= biggest
    full, s2 = serve.serve_gpu(copy.deepcopy(reqs), budget_bytes=10 * biggest, max_slots=5, slice_steps=20,
                               realtime=False)
    assert s2["peak_slots"] > summary["peak_slots"]


def test_channel_bytes_covers_allocation():
    from paper_2108_04435_gb300 import configs, vlb
    for name in ("ring32", "channel64x64x256"):
        p, xyz, nxt = configs.config(name)
        for st in (0, 1):
            p["storage"] = st
            ch = vlb.Channel(p)
            assert vlb.channel_bytes(p) >= ch.stats()[10] > 0
            ch.close()
