"""Seeded synthetic inputs: vortex rings placed in a lattice box.

This module holds no arithmetic of the method; it only lays out filament
points on circles (numpy ``Generator(PCG64(seed))``) so that the CUDA path and
the FP64 oracle start from the same arrays.  The shapes follow the paper's
workloads: single rings (Sec. III.A), ring collisions (Sec. III.B), a
random tangle seeded from rings (Sec. III.C, Sec. IV) and lines bound to the
walls of the closed channel (Sec. IV).
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


def open_line(points):
    """An open line through the given points in order (next = -1 at the last)."""
    xyz = np.asarray(points, np.float64).reshape(-1, 3)
    nxt = np.arange(1, len(xyz) + 1, dtype=np.int32)
    nxt[-1] = -1
    return xyz, nxt


def wall_line(start, end, spacing: float = 0.8):
    """A straight open line from ``start`` to ``end`` (both near walls), with
    equal segments no longer than ``spacing``."""
    a = np.asarray(start, np.float64)
    b = np.asarray(end, np.float64)
    m = max(1, int(np.ceil(np.linalg.norm(b - a) / spacing)))
    t = np.arange(m + 1) / m
    return open_line(a[None, :] + t[:, None] * (b - a)[None, :])


def wall_lines(n_box, count: int, seed: int, amp: float = 0.0, spacing: float = 0.8):
    """``count`` lines along z from the low to the high z wall at random (x, y),
    as in the wall-bound seeds of the closed channel (Sec. IV).  ``amp`` > 0
    adds a helical displacement of that amplitude (one turn along the line),
    vanishing at both walls."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = (float(v) for v in n_box)
    parts = []
    for _ in range(count):
        x0 = rng.uniform(2.0 + amp, nx - 3.0 - amp)
        y0 = rng.uniform(2.0 + amp, ny - 3.0 - amp)
        xyz, nxt = wall_line((x0, y0, 0.0), (x0, y0, nz - 1.0), spacing)
        if amp > 0.0:
            t = (xyz[:, 2] - xyz[0, 2]) / (xyz[-1, 2] - xyz[0, 2])
            env = np.sin(np.pi * t)
            xyz[:, 0] += amp * env * np.cos(2.0 * np.pi * t)
            xyz[:, 1] += amp * env * np.sin(2.0 * np.pi * t)
        parts.append((xyz, nxt))
    return concat(parts)


def concat(parts):
    """Join several (xyz, next) loops or open lines into one point set."""
    xs, ns, off = [], [], 0
    for xyz, nxt in parts:
        nxt = np.asarray(nxt)
        xs.append(xyz)
        ns.append(np.where(nxt >= 0, nxt + off, -1))
        off += len(nxt)
    if not xs:
        return np.zeros((0, 3)), np.zeros(0, np.int32)
    return np.concatenate(xs), np.concatenate(ns).astype(np.int32)


def random_rings(n_box, wall, count: int, r_min: float, r_max: float, seed: int,
                 spacing: float = 0.8, min_sep: float = 2.0, max_tries: int = 200, skip_crowded: bool = False):
    """``count`` rings with radius ~ U[r_min, r_max], random centres and normals.

    Centres are uniform in the box; on wall axes they are kept R + 2 cells
    inside the walls (walls sit half a cell outside the first/last node).  A
    candidate ring that would pass within ``min_sep`` cells of an earlier
    ring is redrawn (intersecting seeds would start from near-singular
    velocities); min_sep = 0 disables the check.  After max_tries the last
    draw is placed anyway, or dropped when skip_crowded is set.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    box = np.asarray(n_box, np.float64)
    periodic = np.array([not w for w in wall])
    grid = _Occupancy(box, periodic, min_sep) if min_sep > 0 else None
    parts = []
    for _ in range(count):
        placed = False
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
            if grid is None or grid.free(xyz):
                placed = True
                break
        if not placed and skip_crowded:
            continue
        parts.append((xyz, nxt))
        if grid is not None:
            grid.add(xyz)
    xyz, nxt = concat(parts)
    for a in range(3):
        if not wall[a]:
            xyz[:, a] = np.mod(xyz[:, a], n_box[a])
    return xyz, nxt


class _Occupancy:
    """Cells of size min_sep/2 within two cells of a placed point.

    A candidate point in a free cell is at least min_sep from every placed
    point (the test is conservative: some farther candidates are refused too).
    """

    def __init__(self, box, periodic, min_sep):
        self.box, self.periodic = box, periodic
        self.h = 0.5 * min_sep
        self.n = np.maximum(np.ceil(box / self.h).astype(int) + 4, 1)
        self.occ = np.zeros(tuple(self.n), dtype=bool)
        self.off = np.array([(i, j, k) for i in range(-2, 3) for j in range(-2, 3) for k in range(-2, 3)])

    def _cells(self, pts):
        q = np.where(self.periodic, np.mod(pts, self.box), pts)
        c = np.floor(q / self.h).astype(int) + 2
        return c

    def _wrap(self, c):
        nper = np.ceil(self.box / self.h).astype(int)
        w = np.where(self.periodic, np.mod(c - 2, nper) + 2, c)
        return np.clip(w, 0, self.n - 1)

    def add(self, pts):
        c = self._cells(pts)
        allc = self._wrap((c[:, None, :] + self.off[None, :, :]).reshape(-1, 3))
        self.occ[allc[:, 0], allc[:, 1], allc[:, 2]] = True

    def free(self, pts):
        c = self._wrap(self._cells(pts))
        return not self.occ[c[:, 0], c[:, 1], c[:, 2]].any()


def perturbed_equilibrium(ncell: int, seed: int, amp: float = 1e-3):
    """Random multiplicative perturbation factors for lattice populations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return 1.0 + amp * rng.uniform(-1.0, 1.0, size=(19, ncell))


def random_field(shape, seed: int, amp: float):
    rng = np.random.Generator(np.random.PCG64(seed))
    return amp * rng.uniform(-1.0, 1.0, size=shape)
