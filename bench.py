"""Benchmark of the coupled vortex-filament / lattice-Boltzmann step.

Metric: coupled-step MLUPS (lattice cells x steps / s of the whole coupled
step) on the closed-channel workload 64x64x256 (walls on all sides, heater
v_n = 0.01, 20 seeded rings, ~1.2k filament points), with filament-point
updates/s beside it.  One process per GPU; with N > 1 every rank runs an
independent replica (the method has no exchange step at one-GPU scale), the
timing is the max over ranks and the value the sum of all ranks' work.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME] [--impl vlb|reference]

--impl reference times the FP64 CPU oracle on this machine's host cores on
the same workload (the reference arm of this benchmark).
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

DEFAULT_CONFIG = "channel64x64x256"
BYTES_PER_CELL = {"f32": 152, "f16": 76, "bf16": 76}  # 19 populations read + 19 written per cell and pass
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}


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
    remesh 2, reconnection 4 = 21.  From 24576 points on the Biot-Savart kernel
    applies the equation of motion itself (17; or as VLB_FUSED_EOM forces)."""
    mode = os.environ.get("VLB_FUSED_EOM")
    fused = n_points >= 24576 if mode is None else mode != "0"
    return 17 if fused else 21


def launches(n_points: int, steps: int, overlap: bool = True) -> int:
    """Kernels of `steps` coupled steps as the library queues them: graphs of
    8 steps while 8 remain, then single steps.  In an 8-step graph the lattice
    passes after the first run alongside the filament chain and write v_n in
    every tile (a memset node sets the tile flags), so 7 tile-flag kernels
    drop out (unless the overlap is off)."""
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
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def k1_traffic(config_name: str):
    """DRAM bytes per stream-collide launch from the committed ncu summary, if
    the kernel source has not changed since it was captured."""
    path = os.path.join(ROOT, "profiles", f"k_lbm_step_{config_name}.md")
    src = os.path.join(ROOT, "paper_2108_04435_gb300", "csrc", "lbm.cu")
    try:
        txt = open(path).read()
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        m = re.search(r"lbm\.cu sha256\[:16\]:\s*([0-9a-f]+)", txt)
        t = re.search(r"dram bytes per launch:\s*([0-9.eE+]+)", txt)
        if m and t and m.group(1) == digest:
            return float(t.group(1))
    except Exception:
        pass
    return None


def run_vlb(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2108_04435_gb300 import configs, vlb

    torch.cuda.set_device(local)
    p, xyz, nxt = configs.config(args.config, seed=rank)
    p["storage"] = STORAGE[args.storage]
    cells = p["n"][0] * p["n"][1] * p["n"][2]
    bpc = BYTES_PER_CELL[args.storage]

    # --- device-resident run: inputs in HBM before the timed region; each step
    # is replayed from the CUDA graph the library captures on first use
    stream = torch.cuda.Stream()
    ch = vlb.Channel(p, stream=stream)
    ch.set_overlap(not args.no_overlap)
    ch.seed(xyz, nxt)
    ch.step(args.warmup)
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
    ch.close()

    # --- the same K steps launched kernel by kernel with CUDA events around
    # every stream-collide launch (graphs off): the roofline of that kernel
    ch = vlb.Channel(p, stream=stream)
    ch.seed(xyz, nxt)
    ch.step(args.warmup)
    ch.set_timing(True)
    torch.cuda.synchronize()
    e0.record(stream)
    ch.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    nograph_s = e0.elapsed_time(e1) / 1e3
    k1_ms, k1_n = ch.lbm_timing()
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
    # vlb_step per step) is timed as well.
    def e2e_run(pipelined):
        ch2 = vlb.Channel(p, stream=stream)
        ch2.set_overlap(not args.no_overlap)
        ch2.step(0)
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ch2.seed(xyz, nxt)
        lengths = []
        if pipelined:
            depth = max(1, min(args.e2e_depth, vlb.ASYNC_DEPTH))
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
    # length among them, and 12 int counters); at the end, the filaments
    d2h = 12 * 8 + 12 * 4 + final.nbytes / args.steps

    pk, pk_kind = peaks()
    k1_avg_s = (k1_ms / 1e3) / max(k1_n, 1)
    achieved = bpc * cells / k1_avg_s / 1e9 if k1_n else None
    traffic = k1_traffic(args.config) if args.storage == "f32" else None
    line = {
        "metric": "coupled-step MLUPS",
        "value": round(mlups, 2),
        "unit": "MLUPS",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(secs * 1e3 / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "storage": args.storage,
        "data": "synthetic (seeded rings, lattice initialised at uniform equilibrium)",
        "config": {"workload": f"{args.config}: D3Q19 {p['n'][0]}x{p['n'][1]}x{p['n'][2]}, walls "
                               f"{tuple(p['wall'])} (1 = bounce-back), heater v_n={p['heater_vn']}, "
                               f"alpha={p['alpha']}, {len(nxt)} seeded filament points on rings",
                   "cells": cells, "filament_points_start": int(len(nxt)),
                   "filament_points_timed": [int(n_before), int(n_after)],
                   "parallelism": f"replicas x{ws}",
                   "l2": l2_note(cells, 4 if args.storage == "f32" else 2)},
        "filament_pts_per_s": round(pts_all / secs, 1),
        "ms_per_step_without_graphs": round(nograph_s * 1e3 / args.steps, 4),
        "e2e": {"value": round(e2e_units / e2e_secs / 1e6, 2), "unit": "MLUPS",
                "h2d_bytes_per_step": round(h2d, 1), "d2h_bytes_per_step": round(d2h, 1),
                "loop": f"vlb_step_async(1) per step, {max(1, min(args.e2e_depth, vlb.ASYNC_DEPTH))} in flight, "
                        "vlb_query + vlb_query_stats per step",
                "blocking_value": round(e2e_block_units / e2e_block_secs / 1e6, 2)},
        # + 1: the line-length kernel that ends each vlb_step call
        "gpu_launches": launches(int(n_before), args.steps, not args.no_overlap) + 1,
        "roofline": {"kernel": "k_lbm_step", "bound": "hbm",
                     "achieved": round(achieved, 1) if achieved else None,
                     "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": round(achieved / pk["hbm_gbs"], 4) if achieved else None,
                     "peak_source": f"{pk_kind} hbm_gbs (copy bandwidth)",
                     "traffic": traffic, "algorithmic_bytes_per_launch": bpc * cells,
                     "avg_launch_us": round(k1_avg_s * 1e6, 3), "launches": k1_n},
        "clocks": clk,
    }
    return line, p, xyz, nxt


def oracle_sample(p, xyz, nxt, budget_s: float, min_steps: int = 2, max_steps: int = 1000):
    """Time the FP64 oracle on host cores for about budget_s seconds."""
    import oracle
    oracle.build()
    ch = oracle.Channel(p)
    ch.seed(xyz, nxt)
    ch.step(1)  # first-touch of the arrays outside the timed part
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps and (steps < min_steps or time.perf_counter() - t0 < budget_s):
        ch.step(1)
        steps += 1
    secs = time.perf_counter() - t0
    n = ch.n_points()
    ch.close()
    cells = p["n"][0] * p["n"][1] * p["n"][2]
    return cells * steps / secs / 1e6, steps, secs, n


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def run_reference(args, ws, rank):
    from paper_2108_04435_gb300 import configs
    if rank != 0:
        return None
    p, xyz, nxt = configs.config(args.config, seed=0)
    import oracle
    oracle.build()
    ch = oracle.Channel(p)
    ch.seed(xyz, nxt)
    ch.step(max(args.warmup, 0))
    t0 = time.perf_counter()
    ch.step(args.steps)
    secs = time.perf_counter() - t0
    cells = p["n"][0] * p["n"][1] * p["n"][2]
    v = cells * args.steps / secs / 1e6
    cores = omp_threads()
    sample = f"{args.steps} full oracle coupled steps of {args.config} after {args.warmup} warm-up steps"
    return {
        "impl": "reference", "metric": "coupled-step MLUPS", "value": round(v, 4), "unit": "MLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "cells": cells},
        "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_serving(args):
    """Sweep of counterflow requests (grids 32^3..128^3, 1.6/1.9/2.1 K,
    v_ns ~ U[0.005, 0.04], 100..20k points) in three forms: the plain FP32
    single-run form (one request at a time, arrivals ignored), and the serving
    form (Poisson arrivals, up to 16 runs admitted by memory budget, steps in
    slices on separate streams) with FP32 and with FP16 population storage."""
    import copy

    from paper_2108_04435_gb300 import configs, serve

    # 16 runs on their own streams: more hardware queues than the default 8
    # (read when the CUDA context is created, so before the first CUDA call)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", str(serve.MAX_CONNECTIONS))
    import torch
    torch.cuda.set_device(0)
    free, total = torch.cuda.mem_get_info()
    budget = int(min(free * 0.8, 64 << 30))
    out = {}
    # sweep throughput: every request available at once
    for form, storage, slots in (("fp32_single_run", 0, 1), ("fp32_serving", 0, 16), ("fp16_serving", 1, 16)):
        reqs = configs.serving_requests(args.requests, args.rate, 0, args.req_steps, storage=storage)
        res, summ = serve.serve_gpu(copy.deepcopy(reqs), budget_bytes=budget, max_slots=slots, slice_steps=50,
                                    realtime=False)
        out[form] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in summ.items()}
    # latency: Poisson arrivals, FP16 serving form
    reqs = configs.serving_requests(args.requests, args.rate, 0, args.req_steps, storage=1)
    res, lat = serve.serve_gpu(copy.deepcopy(reqs), budget_bytes=budget, max_slots=16, slice_steps=50, realtime=True)
    lat = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in lat.items()}
    base = out["fp32_single_run"]["throughput_req_per_s"]
    line = {
        "metric": "serving sweep throughput", "value": out["fp16_serving"]["throughput_req_per_s"],
        "unit": "requests/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "storage": "f16",
        "data": "synthetic",
        "config": {"workload": f"{args.requests} counterflow requests, {args.req_steps} coupled steps each, "
                               f"periodic grids 32^3..128^3, 1.6/1.9/2.1 K",
                   "budget_bytes": budget},
        "speedup_vs_fp32_single_run": round(out["fp16_serving"]["throughput_req_per_s"] / base, 3) if base else None,
        "p50_latency_s": lat["p50_latency_s"], "p99_latency_s": lat["p99_latency_s"],
        "latency_run": {"arrival_rate_per_s": args.rate, **lat},
        "forms": out,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--impl", default="vlb", choices=["vlb", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="population storage (arithmetic is FP32 in all)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--serve", action="store_true", help="serving sweep instead of the coupled-step benchmark")
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--rate", type=float, default=8.0)
    ap.add_argument("--req-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-depth", type=int, default=2,
                    help="one-step calls in flight in the end-to-end loop (1 to 4)")
    ap.add_argument("--no-overlap", action="store_true",
                    help="keep the steps of the 8-step graphs in sequence (vlb_set_overlap off)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_env()
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
        if rank == 0:
            if ws == 1 and not args.no_cpu_baseline:
                v, steps, secs, n = oracle_sample(p, xyz, nxt, args.cpu_budget)
                line["cpu_baseline"] = {"value": round(v, 4), "unit": "MLUPS", "cores": omp_threads(),
                                        "kind": "oracle",
                                        "sample": f"{steps} full FP64 oracle coupled steps of {args.config} from the "
                                                  f"seeded state ({secs:.1f} s)"}
            print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
