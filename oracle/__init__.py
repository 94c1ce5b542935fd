"""FP64 CPU oracle of the coupled VFM-LBM step (arXiv 2108.04435, Sec. II).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers allowed to import this
package.  It shares no code with the CUDA library: its C source
(``vlbref.c``) restates the paper's equations independently, and this module
only marshals arguments through ctypes.

Parity: every function is pinned by the ``-m "not gpu"`` tests against closed
forms, invariants and brute force; see ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vlbref.c")
_LIB = os.path.join(_HERE, "libvlbref.so")
_lock = threading.Lock()
_lib = None

PHASE_LBM, PHASE_VFM, PHASE_REMESH, PHASE_RECONNECT, PHASE_ALL = 1, 2, 4, 8, 15
FIELD_RHO, FIELD_U, FIELD_FSTAR, FIELD_FORCE, FIELD_POS, FIELD_NEXT = 0, 1, 2, 3, 4, 5
FIELD_PLANE_VS, FIELD_STATS, FIELD_VEL, FIELD_ULAST, FIELD_LINE_PROFILE = 6, 7, 8, 9, 10


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "vlbref.h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("n", C.c_int32 * 3), ("wall", C.c_int32 * 3), ("stream_axis", C.c_int32),
        ("vfm_substeps", C.c_int32), ("couple", C.c_int32), ("force_form", C.c_int32),
        ("max_points", C.c_int32), ("reserved", C.c_int32), ("wall_images", C.c_int32), ("reserved2", C.c_int32),
        ("tau", C.c_double), ("rho0", C.c_double), ("body_force", C.c_double * 3),
        ("heater_vn", C.c_double), ("pin_vn", C.c_double), ("init_vn", C.c_double * 3),
        ("kappa", C.c_double), ("alpha", C.c_double), ("alpha_p", C.c_double),
        ("rho_s_over_rho_n", C.c_double), ("core_a", C.c_double),
        ("dxi_min", C.c_double), ("dxi_max", C.c_double),
    ]


def make_params(d: dict) -> Params:
    p = Params()
    for k, v in d.items():
        if k not in dict(Params._fields_):
            continue
        if isinstance(v, (list, tuple)):
            getattr(p, k)[:] = list(v)
        else:
            setattr(p, k, v)
    return p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            _lib.vlbref_create.argtypes = [C.POINTER(Params), C.POINTER(C.c_void_p)]
            _lib.vlbref_destroy.argtypes = [C.c_void_p]
            _lib.vlbref_destroy.restype = None
            _lib.vlbref_last_error.argtypes = [C.c_void_p]
            _lib.vlbref_last_error.restype = C.c_char_p
            _lib.vlbref_seed_vortices.argtypes = [C.c_void_p, dp, ip, C.c_int32]
            _lib.vlbref_step.argtypes = [C.c_void_p, C.c_int32]
            _lib.vlbref_run_phases.argtypes = [C.c_void_p, C.c_int32]
            _lib.vlbref_read_fields.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t,
                                                C.POINTER(C.c_size_t)]
            _lib.vlbref_write_fields.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t]
            _lib.vlbref_line_length.argtypes = [C.c_void_p, dp]
            _lib.vlbref_lattice.argtypes = [ip, dp, ip]
            _lib.vlbref_lattice.restype = None
            _lib.vlbref_feq.argtypes = [C.c_double, dp, dp]
            _lib.vlbref_feq.restype = None
            _lib.vlbref_force_terms.argtypes = [dp, dp, C.c_double, dp]
            _lib.vlbref_force_terms.restype = None
            _lib.vlbref_segment_velocity.argtypes = [dp, dp, dp, C.c_double, dp]
            _lib.vlbref_segment_velocity.restype = None
            _lib.vlbref_geometry.argtypes = [C.c_void_p, dp, dp, dp, dp]
            _lib.vlbref_point_velocity.argtypes = [C.c_void_p, dp, dp]
            _lib.vlbref_interp.argtypes = [C.c_void_p, dp, C.c_int32, dp]
            _lib.vlbref_spread.argtypes = [C.c_void_p, dp, dp, C.c_int32]
        return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class OracleError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"oracle error {code}: {msg}")
        self.code = code


def lattice():
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    lib().vlbref_lattice(_ip(c), _dp(w), _ip(opp))
    return c, w, opp


def feq(rho: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(19)
    lib().vlbref_feq(rho, _dp(u), _dp(out))
    return out


def force_terms(u, F, tau: float) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float64)
    F = np.ascontiguousarray(F, np.float64)
    out = np.zeros(19)
    lib().vlbref_force_terms(_dp(u), _dp(F), tau, _dp(out))
    return out


def segment_velocity(r, s1, s2, kappa: float) -> np.ndarray:
    r, s1, s2 = (np.ascontiguousarray(v, np.float64) for v in (r, s1, s2))
    out = np.zeros(3)
    lib().vlbref_segment_velocity(_dp(r), _dp(s1), _dp(s2), kappa, _dp(out))
    return out


class Channel:
    """One oracle channel: lattice + filaments, host memory, FP64."""

    def __init__(self, params: dict):
        self.params = dict(params)
        self._p = make_params(params)
        h = C.c_void_p()
        rc = lib().vlbref_create(C.byref(self._p), C.byref(h))
        if rc:
            raise OracleError(rc, "create failed")
        self.h = h
        self.n = tuple(int(v) for v in params["n"])
        self.ncell = self.n[0] * self.n[1] * self.n[2]

    def close(self):
        if self.h:
            lib().vlbref_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc:
            raise OracleError(rc, lib().vlbref_last_error(self.h).decode())

    def seed(self, xyz, nxt):
        xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
        nxt = np.ascontiguousarray(nxt, np.int32)
        self._check(lib().vlbref_seed_vortices(self.h, _dp(xyz), _ip(nxt), len(nxt)))

    def step(self, nsteps: int = 1, check: bool = True) -> int:
        rc = lib().vlbref_step(self.h, nsteps)
        if check:
            self._check(rc)
        return rc

    def run_phases(self, mask: int, check: bool = True) -> int:
        rc = lib().vlbref_run_phases(self.h, mask)
        if check:
            self._check(rc)
        return rc

    def n_points(self) -> int:
        return int(self.stats()[0])

    def read(self, which: int) -> np.ndarray:
        N = None
        if which in (FIELD_POS, FIELD_VEL, FIELD_NEXT):
            N = self.n_points()
        shapes = {
            FIELD_RHO: (self.ncell,), FIELD_U: (3, self.ncell), FIELD_FSTAR: (19, self.ncell),
            FIELD_FORCE: (3, self.ncell), FIELD_ULAST: (3, self.ncell),
            FIELD_POS: (N, 3), FIELD_VEL: (N, 3), FIELD_NEXT: (N,),
            FIELD_PLANE_VS: (self.n[self.params.get("stream_axis", 2)],), FIELD_STATS: (16,),
            FIELD_LINE_PROFILE: (self.n[self.params.get("stream_axis", 2)],),
        }
        dtype = np.int32 if which == FIELD_NEXT else np.float64
        out = np.zeros(shapes[which], dtype)
        written = C.c_size_t()
        self._check(lib().vlbref_read_fields(self.h, which, out.ctypes.data_as(C.c_void_p),
                                             out.nbytes, C.byref(written)))
        return out

    def stats(self) -> np.ndarray:
        out = np.zeros(16)
        written = C.c_size_t()
        self._check(lib().vlbref_read_fields(self.h, FIELD_STATS, out.ctypes.data_as(C.c_void_p),
                                             out.nbytes, C.byref(written)))
        return out

    def write(self, which: int, arr: np.ndarray):
        arr = np.ascontiguousarray(arr, np.float64)
        self._check(lib().vlbref_write_fields(self.h, which, arr.ctypes.data_as(C.c_void_p), arr.nbytes))

    def line_length(self) -> float:
        out = C.c_double()
        self._check(lib().vlbref_line_length(self.h, C.byref(out)))
        return out.value

    def geometry(self):
        N = self.n_points()
        sp, spp, lia = np.zeros((N, 3)), np.zeros((N, 3)), np.zeros((N, 3))
        dxi = np.zeros(N)
        self._check(lib().vlbref_geometry(self.h, _dp(sp), _dp(spp), _dp(dxi), _dp(lia)))
        return sp, spp, dxi, lia

    def point_velocity(self):
        N = self.n_points()
        vel, vbs = np.zeros((N, 3)), np.zeros((N, 3))
        self._check(lib().vlbref_point_velocity(self.h, _dp(vel), _dp(vbs)))
        return vel, vbs

    def interp(self, xyz) -> np.ndarray:
        xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
        out = np.zeros_like(xyz)
        self._check(lib().vlbref_interp(self.h, _dp(xyz), len(xyz), _dp(out)))
        return out

    def spread(self, xyz, g):
        xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
        g = np.ascontiguousarray(g, np.float64).reshape(-1, 3)
        self._check(lib().vlbref_spread(self.h, _dp(xyz), _dp(g), len(xyz)))
