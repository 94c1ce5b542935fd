"""Host logic of bench.py: the kernel-launch count it reports as gpu_launches,
and the stream-collide kernel it names in the roofline.

The counts are those of CUPTI traces of the overlapped 8-step graphs
(python -m paper_2108_04435_gb300.trace): 386 kernels for 16 steps of the
64x64x256 channel (1.1k points) and 185 for 8 steps of the 128x128x1024
channel (86k points), each plus the line-length kernel that ends the call."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_launches_per_step(monkeypatch):
    monkeypatch.delenv("VLB_FUSED_EOM", raising=False)
    assert bench.launches_per_step(1148) == 25  # separate equation of motion, point order
    assert bench.launches_per_step(16913) == 28  # + the spatial order
    assert bench.launches_per_step(85770) == 24  # equation of motion inside the Biot-Savart kernel
    monkeypatch.setenv("VLB_FUSED_EOM", "1")
    assert bench.launches_per_step(1148) == 21
    monkeypatch.setenv("VLB_FUSED_EOM", "0")
    assert bench.launches_per_step(85770) == 28
    monkeypatch.setenv("VLB_FUSED_EOM", "00")
    assert bench.launches_per_step(85770) == 28


def test_launches_match_traced_graphs(monkeypatch):
    monkeypatch.delenv("VLB_FUSED_EOM", raising=False)
    assert bench.launches(1148, 16) == 386
    assert bench.launches(85770, 8) == 185
    # without the overlap every step flags its velocity tiles
    assert bench.launches(1148, 16, overlap=False) == 16 * 25
    # single steps after the 8-step graphs
    assert bench.launches(1148, 10) == (8 * 25 - 7) + 2 * 25


def test_stream_collide_kernel_name(monkeypatch):
    monkeypatch.delenv("VLB_LBM_VEC", raising=False)
    assert bench.k1_kernel("f16", 128) == "k_lbm_step_pair"
    assert bench.k1_kernel("bf16", 64) == "k_lbm_step_pair"
    assert bench.k1_kernel("f16", 21) == "k_lbm_step"  # odd nx: one cell per thread
    assert bench.k1_kernel("f32", 128) == "k_lbm_step"
    monkeypatch.setenv("VLB_LBM_VEC", "1")
    assert bench.k1_kernel("f16", 128) == "k_lbm_step"
    # the switch the library ignores leaves its default (4 cells per thread
    # only with FP32 populations, and only where nx divides)
    monkeypatch.setenv("VLB_LBM_VEC", "4")
    assert bench.k1_kernel("f16", 128) == "k_lbm_step_pair"
    assert bench.k1_kernel("f32", 128) == "k_lbm_step_vec"
    assert bench.k1_kernel("f32", 126) == "k_lbm_step"
    monkeypatch.setenv("VLB_LBM_VEC", "2")
    assert bench.k1_kernel("f32", 64) == "k_lbm_step_vec"
    assert bench.k1_kernel("bf16", 21) == "k_lbm_step"
    monkeypatch.setenv("VLB_LBM_VEC", "x")
    assert bench.k1_kernel("f16", 128) == "k_lbm_step_pair"
