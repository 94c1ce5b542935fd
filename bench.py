"""Benchmark of the coupled vortex-filament / lattice-Boltzmann step.

Metric: coupled-step MLUPS (lattice cells x steps / s of the whole coupled
step) on the largest single-GPU workload, the closed channel 128x128x1024
(~16.8M cells, walls on all sides, heater v_n = 0.01, 1.6 K, 1000 seeded
rings of ~86k filament points, FP16 shifted population storage with FP32
arithmetic), with filament-point updates/s beside it.  The line carries the
roofline of the dominant kernel (the Biot-Savart sum, FP32-bound) and of the
stream-collide pass, an end-to-end figure through the C ABI with host
buffers, a short serving sweep with p50/p99 latency, and the FP64 oracle
timed on the host cores.  One process per GPU; with N > 1 every rank runs an
independent replica (the method has no exchange step at one-GPU scale), the
timing is the max over ranks and the value the sum of all ranks' work.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME] [--storage f32|f16|bf16]
                  [--impl vlb|reference] [--serve]

--impl reference times the FP64 CPU oracle on this machine's host cores on
bounded samples of the same workload (the reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_CONFIG = "channel128x128x1024"
DEFAULT_STORAGE = "f16"
BYTES_PER_CELL = {"f32": 152, "f16": 76, "bf16": 76}  # 19 populations read + 19 written per cell and pass
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
# FP32 operations of one (target, segment) pair of the straight-segment
# Biot-Savart formula (Eq. 3): two differences, two norms, the cross and dot
# products, the denominator and three accumulations, with FMA = 2, besides
# 2 reciprocal square roots and 1 reciprocal
BS_FLOP_PER_PAIR = 45
FP32_LANES_PER_SM = 128


def l2_note(cells: int, esize: int) -> str:
    pops = 2 * 19 * esize * cells / 1e6
    fu = (24 + 12) * cells / 1e6  # force grid int64 x 3, velocity float x 3
    rel = "larger" if (pops + fu) > 129.0 else "not larger"
    return (f"working set (2 population buffers {pops:.0f} MB + force/velocity {fu:.0f} MB) {rel} than the "
            f"129 MB L2")


def launches_per_step(n_points: int) -> int:
    """Kernels of one coupled step (1 RK4 sub-step): lattice 3 (velocity-tile
    flags, stream-collide, plane reduction with the force-grid reset),
    filaments 4 x 3 (per RK stage geometry, Biot-Savart, equation of motion),
    remesh 3, reconnection 5 (each ends with the kernel that copies the points
    when its finish changed nothing), and the 2 that assign the Biot-Savart
    source slots once per step = 25.  From 8192 points on, 3 more build the spatial
    order of the sources first; from 24576 points on the Biot-Savart kernel
    applies the equation of motion itself (4 fewer; or as VLB_FUSED_EOM
    forces)."""
    mode = os.environ.get("VLB_FUSED_EOM")
    fused = n_points >= 24576 if mode is None else not mode.startswith("0")  # the library reads the first character
    return (21 if fused else 25) + (3 if n_points >= 8192 else 0)


def launches(n_points: int, steps: int, overlap: bool = True) -> int:
    """Kernels of `steps` coupled steps as the library queues them: graphs of
    8 steps while 8 remain, then single steps.  In an 8-step graph the lattice
    passes after the first run alongside the filament chain and write v_n in
    every tile, so 7 tile-flag kernels drop out (unless the overlap is off)."""
    per = launches_per_step(n_points)
    multi, rest = divmod(steps, 8)
    return multi * (8 * per - (7 if overlap else 0)) + rest * per


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(units: float, seconds: float, ws: int):
    """Sum of work over ranks and max of time over ranks."""
    if ws == 1:
        return units, seconds
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def profile_traffic(kernel: str, config_name: str, sources):
    """DRAM bytes per launch of `kernel` on `config_name` from the committed ncu
    summary profiles/<kernel>_<config>.md, if none of the kernel's source files
    has changed since it was captured (their hash is recorded there)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{config_name}.md")
    h = hashlib.sha256()
    try:
        for src in sources:
            h.update(open(os.path.join(ROOT, "paper_2108_04435_gb300", "csrc", src), "rb").read())
        digest = h.hexdigest()[:16]
        txt = open(path).read()
        m = re.search(r"sources sha256\[:16\]:\s*([0-9a-f]+)", txt)
        t = re.search(r"dram bytes per launch:\s*([0-9.eE+]+)", txt)
        if m and t and m.group(1) == digest:
            return float(t.group(1))
    except Exception:
        pass
    return None


def workload_config(name: str, p: dict, nxt, storage: str, ws: int) -> dict:
    """The `config` object of the JSON line, the same in both arms."""
    cells = p["n"][0] * p["n"][1] * p["n"][2]
    return {"workload": name,
            "description": f"D3Q19 {p['n'][0]}x{p['n'][1]}x{p['n'][2]}, walls {tuple(p['wall'])} "
                           f"(1 = bounce-back), heater v_n={p['heater_vn']}, alpha={p['alpha']}, "
                           f"alpha'={p['alpha_p']}, {len(nxt)} seeded filament points on rings",
            "cells": cells, "filament_points_start": int(len(nxt)), "storage": storage,
            "parallelism": f"replicas x{ws}",
            "l2": l2_note(cells, 4 if storage == "f32" else 2)}


def run_vlb(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2108_04435_gb300 import configs, vlb

    torch.cuda.set_device(local)
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    p, xyz, nxt = configs.config(args.config, seed=rank)
    p["storage"] = STORAGE[args.storage]
    cells = p["n"][0] * p["n"][1] * p["n"][2]
    bpc = BYTES_PER_CELL[args.storage]

    # --- device-resident run: inputs in HBM before the timed region; the steps
    # are replayed from the CUDA graphs the library captures on first use.  The
    # warm-up runs W steps and then the timed call's own step count (twice when
    # it is odd), so that every graph the timed call replays -- the 8-step
    # graphs and the single-step graphs of each buffer parity -- is captured
    # and instantiated before the timer starts.
    stream = torch.cuda.Stream()
    ch = vlb.Channel(p, stream=stream)
    ch.set_overlap(not args.no_overlap)
    ch.seed(xyz, nxt)
    ch.step(args.warmup)
    warm_steps = args.warmup + args.steps
    ch.step(args.steps)
    if args.steps % 2:
        ch.step(args.steps)
        warm_steps += args.steps
    n_before = ch.n_points()
    clocks = ClockSampler(local).start()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ch.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    dev_s = e0.elapsed_time(e1) / 1e3
    n_after = ch.n_points()
    pts = 0.5 * (n_before + n_after) * args.steps  # filament-point updates (mean count x steps)

    # --- the same channel, K more steps launched kernel by kernel with CUDA
    # events on its stream around every stream-collide and Biot-Savart launch
    # (graphs off): the rooflines of the two kernels
    ch.set_timing(True)
    nt0 = ch.n_points()
    torch.cuda.synchronize()
    e0.record(stream)
    ch.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    nograph_s = e0.elapsed_time(e1) / 1e3
    nt1 = ch.n_points()
    k1_ms, k1_n = ch.kernel_timing(vlb.TIMED_LBM)
    bs_ms, bs_n = ch.kernel_timing(vlb.TIMED_BIOT_SAVART)
    ch.set_timing(False)
    ch.close()

    units, secs = aggregate(cells * args.steps, dev_s, ws)
    pts_all, _ = aggregate(pts, dev_s, ws)
    mlups = units / secs / 1e6

    # --- end to end through the public API: seed from host, step one step
    # per call, read every step's status (its line length among it), read
    # the filaments back at the end.  Pipelined: each step is queued with
    # vlb_step_async while the step before still runs, and its status is
    # read once vlb_query has completed it, so the host's launch and read
    # of one step overlap the device's next step.  The blocking loop (one
    # vlb_step per step) is timed as well.  Before the timer, two untimed
    # calls of the same kind capture the graphs the loop replays (both
    # population parities); the filaments are then seeded again inside the
    # timed region.
    def e2e_run(pipelined):
        ch2 = vlb.Channel(p, stream=stream)
        ch2.set_overlap(not args.no_overlap)
        ch2.seed(xyz, nxt)
        depth = max(1, min(args.e2e_depth, vlb.ASYNC_DEPTH))
        if pipelined:
            for _ in range(2):
                ch2.step_async(1)
            for _ in range(2):
                while not ch2.query():
                    pass
        else:
            ch2.step(1)
            ch2.step(1)
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ch2.seed(xyz, nxt)
        lengths = []
        if pipelined:
            for k in range(args.steps + depth - 1):
                if k < args.steps:
                    ch2.step_async(1)
                if k >= depth - 1:
                    while not ch2.query():
                        pass
                    lengths.append(ch2.query_stats()[3])
        else:
            for _ in range(args.steps):
                ch2.step(1)
                lengths.append(ch2.line_length())
        final = ch2.read(vlb.FIELD_POS)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        barrier(ws)
        ch2.close()
        assert len(lengths) == args.steps
        return final, e2e_s

    final, e2e_s = e2e_run(True)
    _, e2e_block_s = e2e_run(False)
    e2e_units, e2e_secs = aggregate(cells * args.steps, e2e_s, ws)
    e2e_block_units, e2e_block_secs = aggregate(cells * args.steps, e2e_block_s, ws)
    h2d = (xyz.size * 8 + nxt.size * 4) / args.steps
    # per step call: the status block (12 doubles of statistics, the line
    # length among them, and 14 int counters); at the end, the filaments
    d2h = 12 * 8 + 14 * 4 + final.nbytes / args.steps

    pk, pk_kind = peaks()
    # stream-collide: algorithmic bytes / mean event-timed launch
    k1_avg_s = (k1_ms / 1e3) / max(k1_n, 1)
    k1_achieved = bpc * cells / k1_avg_s / 1e9 if k1_n else None
    k1_name = k1_kernel(args.storage, p["n"][0])
    k1_traffic = profile_traffic(k1_name, args.config, ["lbm.cu", "vlb_internal.cuh"])
    # Biot-Savart: N (N - 2) pairs per launch at the mean live count of the
    # event-timed steps, 45 FP32 flop each, against the FP32 peak of this
    # GPU (SMs x 128 lanes x 2 flop x clock) at the maximum clock and at the
    # median clock sampled during the timed region
    n_bs = 0.5 * (nt0 + nt1)
    pairs = n_bs * (n_bs - 2)
    bs_avg_s = (bs_ms / 1e3) / max(bs_n, 1)
    bs_tflops = pairs * BS_FLOP_PER_PAIR / bs_avg_s / 1e12 if bs_n else None
    f_max = float(clk.get("sm_max_mhz") or pk.get("sm_max_mhz") or 2070.0)
    f_med = float(clk.get("sm_mhz") or f_max)
    fp32_peak = n_sm * FP32_LANES_PER_SM * 2 * f_max * 1e6 / 1e12
    fp32_peak_med = n_sm * FP32_LANES_PER_SM * 2 * f_med * 1e6 / 1e12
    bs_traffic = profile_traffic("k_biot_savart", args.config, ["bs.cu", "eom.cuh", "records.cuh", "vlb_internal.cuh"])
    bs_share = bs_ms / (nograph_s * 1e3) if nograph_s > 0 else None
    k1_f32 = lbm_pass_roofline(p, "f32", max(10, args.steps), pk, pk_kind, stream) \
        if args.storage != "f32" else None
    k1_alone = lbm_pass_roofline(p, args.storage, max(10, args.steps), pk, pk_kind, stream)
    config = workload_config(args.config, p, nxt, args.storage, ws)
    line = {
        "metric": "coupled-step MLUPS",
        "value": round(mlups, 2),
        "unit": "MLUPS",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "warmup_steps_run": warm_steps,
        "ms_per_step": round(secs * 1e3 / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded rings, lattice initialised at uniform equilibrium)",
        "config": config,
        "filament_points_timed": [int(n_before), int(n_after)],
        "filament_pts_per_s": round(pts_all / secs, 1),
        "ms_per_step_without_graphs": round(nograph_s * 1e3 / args.steps, 4),
        "e2e": {"value": round(e2e_units / e2e_secs / 1e6, 2), "unit": "MLUPS",
                "h2d_bytes_per_step": round(h2d, 1), "d2h_bytes_per_step": round(d2h, 1),
                "loop": f"vlb_step_async(1) per step, {max(1, min(args.e2e_depth, vlb.ASYNC_DEPTH))} in flight, "
                        "vlb_query + vlb_query_stats per step",
                "blocking_value": round(e2e_block_units / e2e_block_secs / 1e6, 2)},
        # + 1: the line-length kernel that ends each vlb_step call
        "gpu_launches": launches(int(n_before), args.steps, not args.no_overlap) + 1,
        "roofline": {"kernel": "k_biot_savart", "bound": "alu",
                     "achieved": round(bs_tflops, 3) if bs_tflops else None,
                     "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                     "frac": round(bs_tflops / fp32_peak, 4) if bs_tflops else None,
                     "peak_source": f"derived FP32 peak: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x "
                                    f"{f_max:.0f} MHz (maximum SM clock)",
                     "frac_at_median_clock": round(bs_tflops / fp32_peak_med, 4) if bs_tflops else None,
                     "median_clock_mhz": f_med,
                     "traffic": bs_traffic,
                     "flop_per_pair": BS_FLOP_PER_PAIR, "pairs_per_launch": round(pairs),
                     "pairs_per_s": round(pairs / bs_avg_s, 1) if bs_n else None,
                     "avg_launch_us": round(bs_avg_s * 1e6, 3), "launches": bs_n,
                     "share_of_event_timed_step": round(bs_share, 4) if bs_share else None},
        "roofline_lbm": {"kernel": k1_name, "bound": "hbm",
                         "achieved": round(k1_achieved, 1) if k1_achieved else None,
                         "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": round(k1_achieved / pk["hbm_gbs"], 4) if k1_achieved else None,
                         "peak_source": f"{pk_kind} hbm_gbs (copy bandwidth)",
                         "traffic": k1_traffic, "algorithmic_bytes_per_launch": bpc * cells,
                         "bytes_per_cell": bpc,
                         "avg_launch_us": round(k1_avg_s * 1e6, 3), "launches": k1_n},
        "clocks": clk,
    }
    line["roofline_lbm_alone"] = k1_alone
    if k1_f32:
        line["roofline_lbm_f32"] = k1_f32
    return line, p, xyz, nxt


def k1_kernel(storage: str, nx: int) -> str:
    """The stream-collide kernel the library launches for this storage and
    x extent, by the library's own rule: two cells per thread with 16-bit
    populations on an even nx, else one; VLB_LBM_VEC (read like C's atoi)
    may ask for 1 or 2 cells per thread, or 4 with FP32 populations, where
    nx divides by it."""
    half = storage != "f32"
    vec = 2 if half and nx % 2 == 0 else 1
    e = os.environ.get("VLB_LBM_VEC")
    if e is not None:
        m = re.match(r"\s*([+-]?\d+)", e)
        v = int(m.group(1)) if m else 0
        if (v in (1, 2) or (v == 4 and not half)) and nx % v == 0:
            vec = v
    if half:
        return "k_lbm_step_pair" if vec == 2 else "k_lbm_step"
    return "k_lbm_step_vec" if vec in (2, 4) else "k_lbm_step"


def lbm_pass_roofline(p, storage, passes, pk, pk_kind, stream):
    """The stream-collide kernel alone on the same grid with another
    population storage: a channel without filaments (so no force or velocity
    tiles flagged), three untimed lattice passes, then `passes` passes with
    CUDA events on the channel's stream around each launch."""
    from paper_2108_04435_gb300 import vlb
    q = dict(p)
    q["storage"] = STORAGE[storage]
    ch = vlb.Channel(q, stream=stream)
    for _ in range(3):
        ch.run_phases(vlb.PHASE_LBM)
    ch.set_timing(True)
    for _ in range(passes):
        ch.run_phases(vlb.PHASE_LBM)
    ms, n = ch.kernel_timing(vlb.TIMED_LBM)
    ch.close()
    cells = q["n"][0] * q["n"][1] * q["n"][2]
    bpc = BYTES_PER_CELL[storage]
    avg_s = ms / 1e3 / max(n, 1)
    achieved = bpc * cells / avg_s / 1e9 if n else None
    return {"kernel": k1_kernel(storage, q["n"][0]), "storage": storage, "bound": "hbm",
            "achieved": round(achieved, 1) if achieved else None, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / pk["hbm_gbs"], 4) if achieved else None,
            "peak_source": f"{pk_kind} hbm_gbs (copy bandwidth)", "traffic": None,
            "algorithmic_bytes_per_launch": bpc * cells, "bytes_per_cell": bpc,
            "avg_launch_us": round(avg_s * 1e6, 3), "launches": n,
            "note": f"lattice passes alone on the benchmark grid (no filaments), populations stored in {storage.upper()}"}


class OracleSampler:
    """The FP64 oracle on host cores, one bounded sample of the workload per
    step, timed; `step_s` is the estimated time of one full oracle coupled step.

    Workloads of up to 8192 filament points run whole oracle coupled steps.
    On larger ones a full oracle step takes minutes (its Biot-Savart sums and
    its brute-force nearest-point search both visit N (N - 2) pairs), so each
    sample step is the oracle's lattice pass over the whole lattice, timed,
    plus its filament phases (RK4 Biot-Savart advance, remesh, reconnection)
    on the first rings of the seed holding about `fil_fraction` of the
    points, timed and scaled by the ratio of the pair counts N (N - 2)."""

    def __init__(self, p, xyz, nxt, fil_fraction: float = 0.125):
        import numpy as np

        import oracle
        oracle.build()
        self.oracle = oracle
        self.cells = p["n"][0] * p["n"][1] * p["n"][2]
        self.n = n = len(nxt)
        self.full = n <= 8192
        nxt = np.asarray(nxt)
        if self.full:
            self.ch = oracle.Channel(p)
            self.ch.seed(xyz, nxt)
            self.ch.step(1)  # first touch of the arrays outside the timed part
            self.m = n
            return
        # the first closed rings (each closes back onto its first point) up to fil_fraction of the points
        ends = [i for i in range(n) if nxt[i] < i]
        self.m = next((e + 1 for e in ends if e + 1 >= fil_fraction * n), n)
        self.lat = oracle.Channel(p)
        self.lat.seed(xyz[:0], nxt[:0])
        self.fil = oracle.Channel(p)
        self.fil.seed(xyz[:self.m], nxt[:self.m])
        self.lat.run_phases(oracle.PHASE_LBM)  # first touch
        self.scale = (n * (n - 2.0)) / (self.m * (self.m - 2.0))

    def step(self):
        """One timed sample step: returns (estimated full-step seconds, lattice s, filament s)."""
        if self.full:
            a = time.perf_counter()
            self.ch.step(1)
            t = time.perf_counter() - a
            return t, t, 0.0
        o = self.oracle
        a = time.perf_counter()
        self.lat.run_phases(o.PHASE_LBM)
        b = time.perf_counter()
        self.fil.run_phases(o.PHASE_VFM | o.PHASE_REMESH | o.PHASE_RECONNECT)
        c = time.perf_counter()
        return (b - a) + (c - b) * self.scale, b - a, c - b

    def describe(self, steps, t_step, t_lat, t_fil):
        if self.full:
            return f"{steps} full FP64 oracle coupled steps ({t_step:.2f} s each)"
        return (f"{steps} sample steps, each the oracle lattice pass over all {self.cells} cells "
                f"({t_lat:.2f} s) + the oracle filament phases on the first {self.m} of {self.n} seeded points "
                f"({t_fil:.2f} s, x{self.scale:.1f} = ratio of N(N-2)); estimated full coupled step {t_step:.1f} s")

    def close(self):
        for name in ("ch", "lat", "fil"):
            if hasattr(self, name):
                getattr(self, name).close()


def oracle_sample(p, xyz, nxt, budget_s: float, min_steps: int = 1, max_steps: int = 1000):
    """Coupled-step MLUPS of the oracle from about budget_s seconds of sample
    steps (OracleSampler), with the description of the sample."""
    smp = OracleSampler(p, xyz, nxt)
    steps, tot, lat, fil, t0 = 0, 0.0, 0.0, 0.0, time.perf_counter()
    while steps < max_steps and (steps < min_steps or time.perf_counter() - t0 < budget_s):
        a, b, c = smp.step()
        tot, lat, fil = tot + a, lat + b, fil + c
        steps += 1
    smp.close()
    step_s = tot / steps
    return smp.cells / step_s / 1e6, smp.describe(steps, step_s, lat / steps, fil / steps), step_s


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def run_reference(args, ws, rank):
    """The reference arm: the FP64 CPU oracle on this machine's host cores.
    Each of the W + K steps is one bounded sample step of the workload
    (OracleSampler), sized so that the whole run ends within a few minutes;
    the value is the coupled-step MLUPS of the K timed samples."""
    from paper_2108_04435_gb300 import configs
    if rank != 0:
        return None
    p, xyz, nxt = configs.config(args.config, seed=0)
    p["storage"] = STORAGE[args.storage]
    cells = p["n"][0] * p["n"][1] * p["n"][2]
    smp = OracleSampler(p, xyz, nxt)
    for _ in range(max(args.warmup, 0)):
        smp.step()
    total_s, lat, fil = 0.0, 0.0, 0.0
    for _ in range(args.steps):
        a, b, c = smp.step()
        total_s, lat, fil = total_s + a, lat + b, fil + c
    smp.close()
    desc = smp.describe(args.steps, total_s / args.steps, lat / args.steps, fil / args.steps)
    v = cells * args.steps / total_s / 1e6
    cores = omp_threads()
    sample = f"{args.config}, after {args.warmup} warm-up sample steps: {desc}"
    return {
        "impl": "reference", "metric": "coupled-step MLUPS", "value": round(v, 4), "unit": "MLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_s * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.config, p, nxt, args.storage, ws),
        "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def serving_sweep(requests: int, rate: float, req_steps: int):
    """Sweep of counterflow requests (grids 32^3..128^3, 1.6/1.9/2.1 K,
    v_ns ~ U[0.005, 0.04], 100..20k points) in three forms: the plain FP32
    single-run form (one request at a time, arrivals ignored), and the serving
    form (up to 16 runs admitted by memory budget, steps in slices on separate
    streams) with FP32 and with FP16 population storage; then the latency of
    the FP16 serving form under Poisson arrivals at `rate`/s.  Failed requests
    are counted in each form with their error messages (CFL: a point moved a
    cell within one step; MACH: |u|/c_s reached 0.05)."""
    import copy

    import torch

    from paper_2108_04435_gb300 import configs, serve

    torch.cuda.set_device(0)
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    budget = int(min(free * 0.8, 64 << 30))
    out = {}
    # sweep throughput: every request available at once
    for form, storage, slots in (("fp32_single_run", 0, 1), ("fp32_serving", 0, 16), ("fp16_serving", 1, 16)):
        reqs = configs.serving_requests(requests, rate, 0, req_steps, storage=storage)
        res, summ = serve.serve_gpu(copy.deepcopy(reqs), budget_bytes=budget, max_slots=slots, slice_steps=50,
                                    realtime=False)
        out[form] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in summ.items()}
    # latency: Poisson arrivals, FP16 serving form
    reqs = configs.serving_requests(requests, rate, 0, req_steps, storage=1)
    res, lat = serve.serve_gpu(copy.deepcopy(reqs), budget_bytes=budget, max_slots=16, slice_steps=50, realtime=True)
    lat = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in lat.items()}
    base = out["fp32_single_run"]["throughput_req_per_s"]
    return {
        "metric": "serving sweep throughput", "value": out["fp16_serving"]["throughput_req_per_s"],
        "unit": "requests/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "storage": "f16",
        "data": "synthetic",
        "config": {"workload": f"{requests} counterflow requests, {req_steps} coupled steps each, "
                               f"periodic grids 32^3..128^3, 1.6/1.9/2.1 K, Poisson arrivals at {rate}/s",
                   "budget_bytes": budget},
        "speedup_vs_fp32_single_run": round(out["fp16_serving"]["throughput_req_per_s"] / base, 3) if base else None,
        "p50_latency_s": lat["p50_latency_s"], "p99_latency_s": lat["p99_latency_s"],
        "failed": {form: out[form]["failed"] for form in out} | {"fp16_serving_poisson": lat["failed"]},
        "latency_run": {"arrival_rate_per_s": rate, **lat},
        "forms": out,
    }


def run_serving(args):
    print(json.dumps(serving_sweep(args.requests, args.rate, args.req_steps)), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--impl", default="vlb", choices=["vlb", "reference"])
    ap.add_argument("--storage", default=DEFAULT_STORAGE, choices=["f32", "f16", "bf16"],
                    help="population storage (arithmetic is FP32 in all)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--serve", action="store_true", help="serving sweep instead of the coupled-step benchmark")
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--rate", type=float, default=8.0)
    ap.add_argument("--req-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving-sample", action="store_true",
                    help="leave out the short serving sweep added to the coupled-step line")
    ap.add_argument("--e2e-depth", type=int, default=2,
                    help="one-step calls in flight in the end-to-end loop (1 to 4)")
    ap.add_argument("--no-overlap", action="store_true",
                    help="keep the steps of the 8-step graphs in sequence (vlb_set_overlap off)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_env()
    if args.serve or (args.impl == "vlb" and ws == 1 and not args.no_serving_sample):
        # many runs on their own streams: more hardware queues than the default
        # 8 (read when the CUDA context is created, so before the first CUDA call)
        from paper_2108_04435_gb300 import serve
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", str(serve.MAX_CONNECTIONS))
    if ws > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.serve:
        if rank == 0:
            run_serving(args)
    elif args.impl == "reference":
        line = run_reference(args, ws, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
    else:
        line, p, xyz, nxt = run_vlb(args, ws, rank, local)
        if rank == 0 and ws == 1:
            if not args.no_serving_sample:
                sv = serving_sweep(args.requests, args.rate, args.req_steps)
                line["serving"] = {k: sv[k] for k in ("value", "unit", "speedup_vs_fp32_single_run", "p50_latency_s",
                                                      "p99_latency_s", "failed", "config")}
                line["serving"]["forms"] = {f: {k: v[k] for k in ("throughput_req_per_s", "mlups", "failed",
                                                                  "failed_ids", "errors", "wall_s")}
                                            for f, v in sv["forms"].items()}
            if not args.no_cpu_baseline:
                v, desc, _ = oracle_sample(p, xyz, nxt, args.cpu_budget)
                line["cpu_baseline"] = {"value": round(v, 4), "unit": "MLUPS", "cores": omp_threads(),
                                        "kind": "oracle", "sample": f"{args.config}: {desc}"}
        if rank == 0:
            print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
