"""The CUPTI kernel-timeline tool (python -m paper_2108_04435_gb300.trace) on a
small workload: every kernel of the step appears, on two streams when the
8-step graphs overlap, and the kernels counted match the launch count the
benchmark reports.  Skipped where CUPTI activity tracing is unavailable."""
import os
import re
import sys

import pytest

pytestmark = pytest.mark.gpu


def test_trace_lists_the_step_kernels(capsys):
    from paper_2108_04435_gb300 import trace
    try:
        trace.main(["--config", "ring32", "--warmup", "8", "--steps", "8"])
    except (OSError, RuntimeError, FileNotFoundError) as e:  # no compiler or no CUPTI here
        pytest.skip(f"CUPTI tracing unavailable: {e}")
    out = capsys.readouterr().out
    for k in ("k_lbm_step", "k_plane_vs", "k_geometry_stage", "k_biot_savart", "k_eom", "k_geometry_exact",
              "k_remesh_finish", "k_hash_insert", "k_nearest", "k_pairs", "k_reconnect_finish", "k_line_length"):
        assert k in out, k
    assert "overlap on" in out
    # the launch count bench.py reports as gpu_launches: 8 steps from one
    # overlapped 8-step graph, then the line-length kernel of the call
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    kernels = int(re.search(r"(\d+) kernels in", out).group(1))
    assert kernels == bench.launches(64, 8, True) + 1, kernels
