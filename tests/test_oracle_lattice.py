"""Pins of the oracle's lattice tables and collision ingredients.

Table I (Sec. II.B) is compared with a text copy of the paper's table; the
equilibrium (Eq. 7) and the forcing term (Eq. 13) are pinned by their moment
identities, which any dropped term, wrong sign or transposed index breaks.
"""
import itertools
import os
import re
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = {}
    for line in open(os.path.join(GOLDEN, "d3q19_table1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w, *pats = line.split()
        vecs = set()
        for pat in pats:
            comps = pat.strip("()").split(",")
            opts = [[s * 1 for s in (1, -1)] if c == "pm1" else [int(c)] for c in comps]
            for v in itertools.product(*opts):
                vecs.add(tuple(v))
        rows[Fraction(w)] = vecs
    return rows


def test_table1_velocity_set_and_weights(oracle_mod):
    c, w, opp = oracle_mod.lattice()
    table = _table1()
    got = {}
    for ci, wi in zip(c, w):
        got.setdefault(Fraction(wi).limit_denominator(100), set()).add(tuple(int(v) for v in ci))
    assert got == table
    assert sum(len(v) for v in table.values()) == 19


def test_opposite_table(oracle_mod):
    c, w, opp = oracle_mod.lattice()
    for i in range(19):
        assert np.array_equal(c[opp[i]], -c[i])
        assert w[opp[i]] == w[i]


def test_isotropy_moments(oracle_mod):
    c, w, _ = oracle_mod.lattice()
    c = c.astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - np.eye(3) / 3).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-16
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.abs(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c) - iso4).max() < 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_feq_moments(oracle_mod, seed):
    """Eq. 7 reproduces rho, rho u and rho (u u + I/3)."""
    rng = np.random.default_rng(seed)
    c, w, _ = oracle_mod.lattice()
    c = c.astype(float)
    rho = 1.0 + 0.1 * rng.uniform(-1, 1)
    u = 0.05 * rng.uniform(-1, 1, 3)
    f = oracle_mod.feq(rho, u)
    assert abs(f.sum() - rho) < 1e-15
    assert np.abs(c.T @ f - rho * u).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ib->ab", f, c, c) - rho * (np.outer(u, u) + np.eye(3) / 3)).max() < 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_force_term_moments(oracle_mod, seed):
    """Eq. 13: zeroth moment 0, first (1 - 1/2tau) F, second (1 - 1/2tau)(uF + Fu)."""
    rng = np.random.default_rng(seed)
    c, w, _ = oracle_mod.lattice()
    c = c.astype(float)
    u = 0.05 * rng.uniform(-1, 1, 3)
    F = 1e-3 * rng.uniform(-1, 1, 3)
    tau = 0.6 + rng.uniform(0, 1)
    Fi = oracle_mod.force_terms(u, F, tau)
    pref = 1.0 - 1.0 / (2.0 * tau)
    assert abs(Fi.sum()) < 1e-18
    assert np.abs(c.T @ Fi - pref * F).max() < 1e-18
    second = np.einsum("i,ia,ib->ab", Fi, c, c)
    assert np.abs(second - pref * (np.outer(u, F) + np.outer(F, u))).max() < 1e-18


def test_unit_conversion_matches_paper():
    """Sec. III: 2 mm over 64 cells, so 0.24 mm is 7.68 cells."""
    from paper_2108_04435_gb300 import configs
    vals = {}
    for line in open(os.path.join(GOLDEN, "paper_units.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    dx_mm = vals["channel_length_mm"] / vals["channel_cells"]
    assert abs(configs.DX_CM * 10.0 - dx_mm) < 1e-15
    assert abs(vals["ring_radius_mm"] / (configs.DX_CM * 10.0) - vals["ring_radius_cells"]) < 1e-12
