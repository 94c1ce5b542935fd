"""The allocation-free Biot-Savart entry point against the allocating one.

vlb_biot_savart_noalloc serves callers that may not allocate device memory
while they run: it keeps its scratch in a fixed device array inside the
library instead of a caller-provided buffer.  Called through the C ABI twice
in a row (the second call reuses the array the first one left behind), it
must give the same velocities as vlb_biot_savart within the tolerance of the
other Biot-Savart tests, from a few hundred points up to its 65536-point
limit (the sizes cover the point-order and the spatially ordered sums).  This
file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(case):
    from paper_2108_04435_gb300 import configs, inputs
    if case == "periodic":
        n, wall = (48, 48, 48), (0, 0, 0)
        xyz, nxt = inputs.random_rings(n, wall, 25, 3.0, 10.0, 11)
    elif case == "walls":
        n, wall = (40, 36, 64), (1, 1, 1)
        xyz, nxt = inputs.random_rings(n, wall, 15, 3.0, 9.0, 12)
    elif case == "sorted-16k":
        n, wall = (128, 128, 128), (0, 0, 0)
        xyz, nxt = inputs.random_rings(n, wall, 170, 6.0, 20.0, 13)
    else:  # "limit": exactly 65536 points in a walled channel
        n, wall = (128, 128, 768), (1, 1, 1)
        xyz, nxt = inputs.random_rings(n, wall, 760, 6.0, 20.0, 14)
        assert len(nxt) >= 65536
        xyz, nxt = xyz[:65536].copy(), np.asarray(nxt[:65536]).copy()
        first = 65535  # the ring cut at the last point closes back onto its own first point
        while first > 0 and nxt[first - 1] == first:
            first -= 1
        nxt[65535] = first
    return configs.base_params(n, wall, 1.9, max_points=8192), xyz, nxt


@pytest.mark.parametrize("case", ["periodic", "walls", "sorted-16k", "limit"])
def test_noalloc_matches_allocating_entry_point(case):
    import torch
    from paper_2108_04435_gb300 import vlb
    p, xyz, nxt = _inputs(case)
    n = len(nxt)
    if case == "limit":
        assert n == 65536
    pos = torch.tensor(np.ascontiguousarray(np.asarray(xyz).T), dtype=torch.float64, device="cuda")
    nx = torch.tensor(np.asarray(nxt, np.int32), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.zeros((3, n), dtype=torch.float32, device="cuda")
    sb = vlb.biot_savart_scratch_bytes(n)
    scratch = torch.empty(sb, dtype=torch.uint8, device="cuda")
    vlb.biot_savart(p, pos.data_ptr(), nx.data_ptr(), n, ref.data_ptr(), scratch.data_ptr(), sb, stream)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy().astype(np.float64)
    for _ in range(2):
        out = torch.full((3, n), float("nan"), dtype=torch.float32, device="cuda")
        vlb.biot_savart_noalloc(p, pos.data_ptr(), nx.data_ptr(), n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_noalloc_rejects_too_many_points():
    from paper_2108_04435_gb300 import configs, vlb
    p = configs.base_params((32, 32, 32), (0, 0, 0), 1.9)
    with pytest.raises(vlb.VlbError) as e:
        vlb.biot_savart_noalloc(p, 1, 1, 65537, 1, 0)
    assert e.value.code == -1
