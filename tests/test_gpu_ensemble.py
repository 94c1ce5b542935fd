"""Long runs: GPU (FP32) against the FP64 oracle on ensemble statistics.

Per-step parity holds from identical states; over long runs filaments and
reconnection decisions drift apart chaotically, so the two are compared on
the ensemble quantities the method is used for: the vortex line length
(line density, Sec. III.C) and the plane-mean normal-velocity profile
(Eq. 18), each to 2%, over several seeds of a counterflow tangle."""
import numpy as np
import pytest

from gpu_util import pair

pytestmark = pytest.mark.gpu


def test_counterflow_tangle_ensemble():
    import oracle
    from paper_2108_04435_gb300 import configs, inputs, vlb
    n, wall = (32, 32, 32), (0, 0, 0)
    lengths_g, lengths_r, prof_g, prof_r = [], [], [], []
    for seed in range(3):
        xyz, nxt = inputs.random_rings(n, wall, 6, 4.0, 8.0, 100 + seed)
        p = configs.base_params(n, wall, 1.9, max_points=4096,
                                init_vn=[0.0, 0.0, configs.counterflow_vn(0.02, 1.9)])
        g, r = pair(p, xyz, nxt)
        g.step(300)
        r.step(300)
        lengths_g.append(g.line_length())
        lengths_r.append(r.line_length())
        prof_g.append(g.read(vlb.FIELD_U)[2].reshape(n[2], -1).mean(axis=1))
        prof_r.append(r.read(oracle.FIELD_U)[2].reshape(n[2], -1).mean(axis=1))
        g.close()
    Lg, Lr = np.mean(lengths_g), np.mean(lengths_r)
    assert abs(Lg / Lr - 1) < 0.02, (lengths_g, lengths_r)
    pg, pr = np.mean(prof_g, axis=0), np.mean(prof_r, axis=0)
    assert np.abs(pg - pr).max() < 0.02 * np.abs(pr).mean()
