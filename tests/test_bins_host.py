"""Host logic of the spatial order of the Biot-Savart sources (no GPU): the
bins the library chooses for a lattice, compiled from its own header by nvcc
as host code and run on the CPU.

For every lattice: the Morton key of a bin has at most 8 bits (K = 2^bits <=
256 bins), every cell's bin index fits its axis' bits, bins are 16 cells wide
or more and the widest of 64, 32 and 16 that still leaves 64 bins (wider only
to fit 8 bits), and the per-block bin counts of the sort (K per 1024 points)
fit in the cap ints of their buffer from the sort's 8192 points on."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2108_04435_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "vlb_internal.cuh"
int main() {
    const int ns[] = {1, 2, 5, 16, 17, 31, 32, 33, 64, 100, 128, 255, 256, 257, 1000, 1024, 2048, 4096};
    for (int a : ns) for (int b : ns) for (int c : ns) {
        const vlb::BsBins bb = vlb::bs_bins(a, b, c);
        std::printf("%d %d %d %d %d %d %d %d\n", a, b, c, bb.shift, bb.bits[0], bb.bits[1], bb.bits[2], bb.K);
    }
    std::printf("MIN %d MAXBINS %d\n", vlb::BS_SORT_MIN, vlb::BS_SORT_MAX_BINS);
    return 0;
}
"""


@pytest.fixture(scope="module")
def bins(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("bins")
    src, exe = d / "bins.cu", d / "bins"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)], check=True,
                   capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split("\n")
    rows = [tuple(map(int, line.split())) for line in out if line and not line.startswith("MIN")]
    tail = [line.split() for line in out if line.startswith("MIN")][0]
    return rows, int(tail[1]), int(tail[3])


def ceil_div(a, b):
    return (a + b - 1) // b


def test_bins_fit_eight_bit_keys(bins):
    rows, _, max_bins = bins
    for a, b, c, shift, bx, by, bz, K in rows:
        assert bx + by + bz <= 8 and K == 1 << (bx + by + bz) and K <= max_bins <= 256
        e = 1 << shift
        for n, bits in ((a, bx), (b, by), (c, bz)):
            # the highest bin index of the axis, (n - 1) >> shift, fits its bits
            assert ((n - 1) >> shift) < (1 << bits), (a, b, c)
            assert ceil_div(n, e) <= 1 << bits


def test_bins_are_the_widest_that_leave_64(bins):
    rows, _, _ = bins
    for a, b, c, shift, bx, by, bz, K in rows:
        count = lambda s: ceil_div(a, 1 << s) * ceil_div(b, 1 << s) * ceil_div(c, 1 << s)  # noqa: E731
        key_bits = lambda s: sum((ceil_div(n, 1 << s) - 1).bit_length() for n in (a, b, c))  # noqa: E731
        # the widest of 64, 32, 16 cells that leaves 64 bins (16 if none does)
        first = next((s for s in (6, 5) if count(s) >= 64), 4)
        assert shift >= first, (a, b, c)
        # widened from there only as far as 8 key bits need
        assert key_bits(shift) <= 8
        if shift > first:
            assert key_bits(shift - 1) > 8, (a, b, c)


def test_benchmark_lattices(bins):
    rows, _, _ = bins
    got = {(r[0], r[1], r[2]): (r[3], r[7]) for r in rows}
    assert got[(128, 128, 1024)] == (6, 64)    # 2 x 2 x 16 bins of 64 cells
    assert got[(128, 128, 128)] == (5, 64)     # 4 x 4 x 4 bins of 32 cells
    assert got[(64, 64, 256)] == (4, 256)      # 4 x 4 x 16 bins of 16 cells
    assert got[(1024, 1024, 1024)] == (8, 64)  # 64-cell bins need 12 bits, 128-cell 9: 4^3 of 256 cells


def test_sort_counts_fit_their_buffer(bins):
    _, sort_min, max_bins = bins
    for cap in list(range(sort_min, 70000, 997)) + [sort_min, 262144, 1 << 22]:
        assert max_bins * ceil_div(cap, 1024) <= cap
