"""Serving loop: counterflow runs admitted as they arrive, batched on one GPU.

Requests (a lattice, a temperature, a counterflow, seeded filaments and a
number of coupled steps) arrive over time.  The loop admits a waiting request
as soon as a slot and enough of the device-memory budget are free, gives it a
channel on its own CUDA stream (state stays resident until the request
finishes) and keeps every admitted run busy with slices of graph-replayed
steps queued with vlb_step_async.  Runs on different streams overlap on the
GPU; a slow run never blocks a fast one.  Latency is arrival to completion,
queueing included.

All device work is done by libvlb through its C ABI; this module only
schedules.  `Scheduler` holds the admission and bookkeeping logic and is
independent of the GPU (it takes a factory for the run objects).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Result:
    id: int
    arrival: float
    start: float = 0.0
    finish: float = 0.0
    steps: int = 0
    cells: int = 0
    points_mean: float = 0.0
    line_length: float = 0.0
    n_points: int = 0
    error: str = ""
    state: dict = field(default_factory=dict)  # fields read at completion (serve_gpu's snapshot)

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


@dataclass
class _Active:
    req: dict
    run: object
    res: Result
    remaining: int
    bytes: int
    pts_sum: float = 0.0
    slices: int = 0


@dataclass
class Scheduler:
    """Admission by slots and memory budget; slices of steps per admitted run.

    make_run(req) -> object with step_async(n), query() -> bool, n_points(),
    line_length(), close(); bytes_of(req) -> int.
    """
    make_run: object
    bytes_of: object
    budget_bytes: int
    max_slots: int = 16
    slice_steps: int = 50
    clock: object = time.perf_counter
    results: list = field(default_factory=list)
    peak_bytes: int = 0
    peak_slots: int = 0

    def serve(self, requests, realtime: bool = True, idle_sleep: float = 0.0002):
        pending = sorted(requests, key=lambda r: r["arrival"])
        waiting, active = [], []
        used = 0
        t0 = self.clock()
        i = 0
        while i < len(pending) or waiting or active:
            now = self.clock() - t0
            while i < len(pending) and (not realtime or pending[i]["arrival"] <= now):
                waiting.append(pending[i])
                i += 1
            # admit in arrival order while a slot and the memory are free
            while waiting and len(active) < self.max_slots:
                need = self.bytes_of(waiting[0])
                if used + need > self.budget_bytes and active:
                    break
                req = waiting.pop(0)
                res = Result(id=req["id"], arrival=req["arrival"] if realtime else 0.0, start=self.clock() - t0)
                try:
                    run = self.make_run(req)
                except Exception as e:  # a request that cannot be created is reported, not retried
                    res.error = str(e)
                    res.finish = self.clock() - t0
                    self.results.append(res)
                    continue
                n0 = run.n_points()
                a = _Active(req=req, run=run, res=res, remaining=req["steps"], bytes=need, pts_sum=0.0)
                a.pts_sum += n0
                used += need
                active.append(a)
                run.step_async(min(self.slice_steps, a.remaining))
            self.peak_bytes = max(self.peak_bytes, used)
            self.peak_slots = max(self.peak_slots, len(active))
            progressed = False
            for a in list(active):
                try:
                    if not a.run.query():
                        continue
                except Exception as e:
                    a.res.error = str(e)
                    a.remaining = 0
                progressed = True
                done = min(self.slice_steps, a.remaining)
                a.remaining -= done
                a.res.steps += done
                a.slices += 1
                if a.remaining > 0:
                    a.pts_sum += a.run.n_points()
                    a.run.step_async(min(self.slice_steps, a.remaining))
                    continue
                a.res.finish = self.clock() - t0
                if not a.res.error:
                    a.res.n_points = a.run.n_points()
                    a.res.line_length = a.run.line_length()
                    if hasattr(a.run, "final_state"):
                        a.res.state = a.run.final_state()
                a.res.points_mean = a.pts_sum / max(1, a.slices)
                a.run.close()
                used -= a.bytes
                active.remove(a)
                self.results.append(a.res)
            if not progressed and idle_sleep:
                time.sleep(idle_sleep)
        return sorted(self.results, key=lambda r: r.id)


def summarize(results, wall_s: float):
    ok = [r for r in results if not r.error]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    cells_steps = sum(r.cells * r.steps for r in ok)
    pts_steps = sum(r.points_mean * r.steps for r in ok)
    return {
        "requests": len(results), "failed": len(results) - len(ok),
        "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
        "throughput_req_per_s": len(ok) / wall_s, "mlups": cells_steps / wall_s / 1e6,
        "filament_pts_per_s": pts_steps / wall_s, "wall_s": wall_s,
        "errors": sorted({r.error for r in results if r.error})[:5],
        "failed_ids": [r.id for r in results if r.error],
    }


# Hardware work queues for a serving process (CUDA_DEVICE_MAX_CONNECTIONS).
MAX_CONNECTIONS = 32


class GpuRun:
    """One request as a libvlb channel on its own stream.  With other runs
    sharing the GPU (overlap=False) the channel keeps its steps in sequence:
    the runs overlap one another already, and a second stream per channel
    would compete for the device's hardware queues."""

    def __init__(self, req, device: int = 0, overlap: bool = True, snapshot=()):
        import torch

        from . import vlb
        self.ch = vlb.Channel(req["params"], stream=torch.cuda.Stream(device), device=device)
        self.ch.set_overlap(overlap)
        self.ch.seed(req["xyz"], req["next"])
        self._n = len(req["next"])
        self.snapshot = tuple(snapshot)

    def final_state(self):
        """The fields named in `snapshot` (vlb.FIELD_*), read at completion."""
        return {w: self.ch.read(w) for w in self.snapshot}

    def step_async(self, n):
        self.ch.step_async(n)

    def query(self):
        return self.ch.query()

    def n_points(self):
        return self.ch.n_points()

    def line_length(self):
        return self.ch.line_length()

    def close(self):
        self.ch.close()


def serve_gpu(requests, budget_bytes: int, max_slots: int = 16, slice_steps: int = 50, realtime: bool = True,
              snapshot=()):
    """Serve requests on the current GPU; returns (results, summary).  Many
    channels on their own streams share the device's hardware work queues
    (8 unless CUDA_DEVICE_MAX_CONNECTIONS, read when the process creates its
    CUDA context, says otherwise); MAX_CONNECTIONS is the value to set before
    that for 16 slots.  `snapshot` names fields (vlb.FIELD_*) to read from
    each run when it completes, into its Result.state."""
    from . import vlb
    for r in requests:
        n = r["params"]["n"]
        r.setdefault("cells", n[0] * n[1] * n[2])
    make = lambda req: GpuRun(req, overlap=max_slots == 1, snapshot=snapshot)  # noqa: E731
    sched = Scheduler(make_run=make, bytes_of=lambda r: vlb.channel_bytes(r["params"]), budget_bytes=budget_bytes,
                      max_slots=max_slots, slice_steps=slice_steps)
    t0 = time.perf_counter()
    res = sched.serve(requests, realtime=realtime)
    wall = time.perf_counter() - t0
    for r in res:
        r.cells = next(q["cells"] for q in requests if q["id"] == r.id)
    summary = summarize(res, wall)
    summary.update(peak_slots=sched.peak_slots, peak_bytes=sched.peak_bytes)
    return res, summary
