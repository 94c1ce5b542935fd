"""Kernel timeline of coupled steps from CUPTI activity records.

    python -m paper_2108_04435_gb300.trace [--config NAME] [--storage f32|f16|bf16] [--warmup 16] [--steps 16] [--no-overlap]

Runs `warmup` steps, then records the start and end of every kernel of
`steps` more (replayed from the 8-step graphs when steps is a multiple of 8)
and prints per-kernel means and the two-stream timeline of the last full
step: the overlap of the lattice pass with the filament chain that ncu, which
serialises graph nodes, cannot show.  The CUPTI shim (csrc/trace.cpp) is
compiled on first use with the host compiler; it is a profiling aid, not part
of the step.
"""
from __future__ import annotations

import argparse
import ctypes as C
import os
import re
import subprocess
import sys
import tempfile
from collections import defaultdict

HERE = os.path.dirname(os.path.abspath(__file__))


def tracer() -> C.CDLL:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    src = os.path.join(HERE, "csrc", "trace.cpp")
    out = os.path.join(HERE, "_build", "libvlbtrace.so")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        subprocess.run(["g++", "-O2", "-shared", "-fPIC", src, "-I" + os.path.join(cuda, "include"),
                        "-L" + os.path.join(cuda, "lib64"), "-lcupti", "-o", out], check=True)
    lib = C.CDLL(out)
    lib.trace_stop.argtypes = [C.c_char_p]
    return lib


def short(name: str) -> str:
    m = re.search(r"(k_[a-z_0-9]+)", name)
    return m.group(1) if m else name.strip()


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="channel64x64x256")
    ap.add_argument("--warmup", type=int, default=16)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--no-overlap", action="store_true")
    ap.add_argument("--storage", choices=("f32", "f16", "bf16"), default=None,
                    help="population storage (default: the configuration's)")
    a = ap.parse_args(argv)
    lib = tracer()
    import torch

    from . import configs, vlb
    p, xyz, nxt = configs.config(a.config)
    if a.storage:
        p["storage"] = {"f32": 0, "f16": 1, "bf16": 2}[a.storage]
    ch = vlb.Channel(p)
    ch.set_overlap(not a.no_overlap)
    ch.seed(xyz, nxt)
    ch.step(a.warmup)
    torch.cuda.synchronize()
    if lib.trace_start() != 0:
        raise RuntimeError("CUPTI activity tracing could not be enabled")
    ch.step(a.steps)
    torch.cuda.synchronize()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "trace.txt")
        lib.trace_stop(path.encode())
        rows = []
        for line in open(path):
            s, e, st, nm = line.split(None, 3)
            rows.append((int(s), int(e), int(st), short(nm)))
    ch.close()
    rows.sort()
    t0 = rows[0][0]
    span = (rows[-1][1] - t0) / 1e3
    streams = sorted({r[2] for r in rows})
    print(f"{a.config}: {a.steps} steps after {a.warmup}, overlap {'off' if a.no_overlap else 'on'}; "
          f"{len(rows)} kernels in {span:.1f} us ({span / a.steps:.1f} us per step)")
    tot, cnt = defaultdict(float), defaultdict(int)
    for s, e, st, nm in rows:
        tot[nm] += (e - s) / 1e3
        cnt[nm] += 1
    print(f"\n{'kernel':24s} {'launches':>8s} {'mean us':>8s} {'total us':>9s}")
    for nm in sorted(tot, key=lambda k: -tot[k]):
        print(f"{nm:24s} {cnt[nm]:8d} {tot[nm] / cnt[nm]:8.2f} {tot[nm]:9.1f}")
    # about the last two steps' records
    tail = rows[-max(1, 2 * len(rows) // a.steps):]
    base = tail[0][0]
    print("\ntimeline of the last two steps (start and duration in us; one column per stream)")
    for s, e, st, nm in tail:
        print(f"{'    ' * streams.index(st)}{nm:24s} start {(s - base) / 1e3:8.2f}  dur {(e - s) / 1e3:6.2f}")


if __name__ == "__main__":
    main(sys.argv[1:])
