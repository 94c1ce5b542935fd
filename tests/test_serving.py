"""Serving scheduler (host logic, no GPU): admission by slots and by the
device-memory budget, arrival-order admission, slices of steps until each
request has run all its steps."""

from paper_2108_04435_gb300.serve import Scheduler, summarize


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


class FakeRun:
    live = 0
    peak = 0

    def __init__(self, req):
        self.req = req
        self.busy = 0
        FakeRun.live += 1
        FakeRun.peak = max(FakeRun.peak, FakeRun.live)

    def step_async(self, n):
        self.busy = 3  # finished after three polls

    def query(self):
        self.busy -= 1
        return self.busy <= 0

    def n_points(self):
        return 10

    def line_length(self):
        return float(self.req["id"])

    def close(self):
        FakeRun.live -= 1


def make_requests(n, steps):
    return [dict(id=k, arrival=0.01 * k, steps=steps, size=100 + 50 * (k % 3)) for k in range(n)]


def test_slots_budget_and_completion():
    FakeRun.live = FakeRun.peak = 0
    reqs = make_requests(12, 130)
    s = Scheduler(make_run=FakeRun, bytes_of=lambda r: r["size"], budget_bytes=400, max_slots=3, slice_steps=50,
                  clock=FakeClock())
    res = s.serve(reqs, realtime=True, idle_sleep=0)
    assert [r.id for r in res] == list(range(12))
    assert all(r.steps == 130 and not r.error for r in res)
    assert FakeRun.peak <= 3 and s.peak_slots <= 3
    assert s.peak_bytes <= 400
    assert all(r.line_length == r.id for r in res)
    assert all(r.finish >= r.start >= r.arrival for r in res)


def test_admission_in_arrival_order_when_full():
    reqs = make_requests(6, 50)
    order = []

    def make(req):
        order.append(req["id"])
        return FakeRun(req)

    s = Scheduler(make_run=make, bytes_of=lambda r: 1, budget_bytes=10, max_slots=1, slice_steps=50,
                  clock=FakeClock())
    s.serve(reqs, realtime=False, idle_sleep=0)
    assert order == list(range(6))


def test_summary_percentiles():
    from paper_2108_04435_gb300.serve import Result
    res = [Result(id=k, arrival=0.0, start=0.0, finish=float(k + 1), steps=10, cells=100) for k in range(100)]
    s = summarize(res, wall_s=10.0)
    assert abs(s["p50_latency_s"] - 50.5) < 1e-9 and abs(s["p99_latency_s"] - 99.01) < 1e-9
    assert s["mlups"] == 100 * 10 * 100 / 10.0 / 1e6


def test_summary_counts_only_completed_requests():
    # a failed request (CFL or Mach check) is listed, not counted in
    # throughput, latency or lattice updates
    from paper_2108_04435_gb300.serve import Result
    res = [Result(id=k, arrival=0.0, finish=2.0, steps=10, cells=100) for k in range(4)]
    res[1].error = "VLB_ERR_CFL: a filament point moved a cell within a step"
    res[3].error = "VLB_ERR_MACH: lattice velocity exceeds the Mach limit"
    res[3].finish = 100.0
    s = summarize(res, wall_s=4.0)
    assert s["requests"] == 4 and s["failed"] == 2 and s["failed_ids"] == [1, 3]
    assert s["throughput_req_per_s"] == 2 / 4.0
    assert s["mlups"] == 2 * 100 * 10 / 4.0 / 1e6
    assert s["p99_latency_s"] == 2.0
    assert len(s["errors"]) == 2
