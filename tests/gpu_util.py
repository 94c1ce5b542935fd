"""Helpers for the GPU parity tests: both sides from the same seeded arrays."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def pair(params, xyz=None, nxt=None):
    """A GPU channel and an oracle channel with the same parameters and filaments."""
    import oracle
    from paper_2108_04435_gb300 import vlb
    g = vlb.Channel(params)
    r = oracle.Channel(params)
    if xyz is not None:
        g.seed(xyz, nxt)
        r.seed(xyz, nxt)
    return g, r


def same_lattice_state(g, r, seed, amp=1e-2, force_amp=0.0):
    """Perturb the populations (and optionally the force grid) identically on both sides.
    The GPU stores float32, so the oracle receives the float32-rounded values."""
    import oracle
    from paper_2108_04435_gb300 import inputs, vlb
    f0 = r.read(oracle.FIELD_FSTAR)
    f = (f0 * inputs.perturbed_equilibrium(r.ncell, seed, amp)).astype(np.float32)
    g.write(vlb.FIELD_FSTAR, f)
    r.write(oracle.FIELD_FSTAR, f.astype(np.float64))
    if force_amp > 0:
        F = inputs.random_field((3, r.ncell), seed + 1, force_amp).astype(np.float32)
        g.write(vlb.FIELD_FORCE, F)
        r.write(oracle.FIELD_FORCE, F.astype(np.float64))
    return f
