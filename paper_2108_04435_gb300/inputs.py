"""Seeded synthetic inputs: vortex rings placed in a lattice box.

This module holds no arithmetic of the method; it only lays out filament
points on circles (numpy ``Generator(PCG64(seed))``) so that the CUDA path and
the FP64 oracle start from the same arrays.  The shapes follow the paper's
workloads: single rings (Sec. III.A), ring collisions (Sec. III.B) and a
random tangle seeded from rings (Sec. III.C, Sec. IV).
"""
from __future__ import annotations

import numpy as np


def ring(center, normal, radius: float, npts: int | None = None, spacing: float = 0.8,
         phase: float = 0.0):
    """Points on a circle, ordered counter-clockwise about ``normal``.

    Returns (xyz [n,3] float64, next [n] int32).  With that ordering the ring's
    self-induced motion is along +normal.
    """
    c = np.asarray(center, np.float64)
    n = np.asarray(normal, np.float64)
    n = n / np.linalg.norm(n)
    ref = np.array([1.0, 0.0, 0.0]) if abs(n[0]) <= 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(n, ref)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    if npts is None:
        npts = max(5, int(round(2.0 * np.pi * radius / spacing)))
    th = phase + 2.0 * np.pi * np.arange(npts) / npts
    xyz = c[None, :] + radius * (np.cos(th)[:, None] * e1[None, :] + np.sin(th)[:, None] * e2[None, :])
    nxt = ((np.arange(npts) + 1) % npts).astype(np.int32)
    return xyz, nxt


def concat(parts):
    """Join several (xyz, next) loops into one point set."""
    xs, ns, off = [], [], 0
    for xyz, nxt in parts:
        xs.append(xyz)
        ns.append(nxt + off)
        off += len(nxt)
    if not xs:
        return np.zeros((0, 3)), np.zeros(0, np.int32)
    return np.concatenate(xs), np.concatenate(ns).astype(np.int32)


def random_rings(n_box, wall, count: int, r_min: float, r_max: float, seed: int,
                 spacing: float = 0.8, min_sep: float = 2.0, max_tries: int = 200):
    """``count`` rings with radius ~ U[r_min, r_max], random centres and normals.

    Centres are uniform in the box; on wall axes they are kept R + 2 cells
    inside the walls (walls sit half a cell outside the first/last node).  A
    candidate ring that would pass within ``min_sep`` cells of an earlier
    ring is redrawn (intersecting seeds would start from near-singular
    velocities); min_sep = 0 disables the check.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    box = np.asarray(n_box, np.float64)
    periodic = np.array([not w for w in wall])
    grid = _PointGrid(box, periodic, max(min_sep, 1e-9))
    parts = []
    for _ in range(count):
        for _try in range(max_tries):
            R = rng.uniform(r_min, r_max)
            c = np.empty(3)
            for a in range(3):
                if wall[a]:
                    lo, hi = -0.5 + R + 2.0, n_box[a] - 0.5 - R - 2.0
                    if hi <= lo:
                        raise ValueError("box too small for ring radius")
                    c[a] = rng.uniform(lo, hi)
                else:
                    c[a] = rng.uniform(0.0, n_box[a])
            nrm = rng.normal(size=3)
            nrm /= np.linalg.norm(nrm)
            phase = rng.uniform(0.0, 2.0 * np.pi)
            xyz, nxt = ring(c, nrm, R, spacing=spacing, phase=phase)
            if min_sep <= 0 or grid.clearance(xyz, min_sep) >= min_sep:
                break
        parts.append((xyz, nxt))
        grid.add(xyz)
    xyz, nxt = concat(parts)
    for a in range(3):
        if not wall[a]:
            xyz[:, a] = np.mod(xyz[:, a], n_box[a])
    return xyz, nxt


class _PointGrid:
    """Uniform grid of cell size h over placed points, for clearance queries."""

    def __init__(self, box, periodic, h):
        self.box, self.periodic, self.h = box, periodic, h
        self.ncell = np.maximum(np.floor(box / h).astype(int), 1)
        self.cells = {}

    def _key(self, c):
        c = np.where(self.periodic, np.mod(c, self.ncell), c)
        return tuple(int(v) for v in c)

    def _cells_of(self, pts):
        return np.floor(np.where(self.periodic, np.mod(pts, self.box), pts) / self.h).astype(int)

    def add(self, pts):
        for q, c in zip(pts, self._cells_of(pts)):
            self.cells.setdefault(self._key(c), []).append(q)

    def clearance(self, pts, stop_below=0.0):
        """Smallest distance from pts to the placed points (stops early below stop_below)."""
        best = np.inf
        if not self.cells:
            return best
        offs = [(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)]
        for q, c in zip(pts, self._cells_of(pts)):
            for o in offs:
                lst = self.cells.get(self._key(c + np.array(o)))
                if not lst:
                    continue
                d = np.asarray(lst) - q
                d = np.where(self.periodic, d - self.box * np.round(d / self.box), d)
                best = min(best, float(np.sqrt((d * d).sum(-1)).min()))
                if best < stop_below:
                    return best
        return best


def perturbed_equilibrium(ncell: int, seed: int, amp: float = 1e-3):
    """Random multiplicative perturbation factors for lattice populations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return 1.0 + amp * rng.uniform(-1.0, 1.0, size=(19, ncell))


def random_field(shape, seed: int, amp: float):
    rng = np.random.Generator(np.random.PCG64(seed))
    return amp * rng.uniform(-1.0, 1.0, size=shape)
