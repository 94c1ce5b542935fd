"""ctypes binding of libvlb.so (the C ABI in include/vlb.h).

Argument marshalling only: every step of the coupled update runs in the CUDA
kernels behind the C ABI.  PyTorch supplies device memory (its caching
allocator, through the ABI's allocator callbacks) and the stream.  There is no
fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvlb.so")

OK = 0
ERR = {-1: "INVALID_ARG", -2: "OOM", -3: "CAPACITY", -4: "TOPOLOGY", -5: "MACH", -6: "NAN",
       -7: "TIMEOUT", -8: "CUDA", -9: "CFL"}
PHASE_LBM, PHASE_VFM, PHASE_REMESH, PHASE_RECONNECT, PHASE_ALL = 1, 2, 4, 8, 15
FIELD_RHO, FIELD_U, FIELD_FSTAR, FIELD_FORCE, FIELD_POS, FIELD_NEXT = 0, 1, 2, 3, 4, 5
FIELD_PLANE_VS, FIELD_STATS, FIELD_VEL, FIELD_FDEV, FIELD_LINE_PROFILE = 6, 7, 8, 9, 10

EXPORTS = ["vlb_create_channel", "vlb_seed_vortices", "vlb_step", "vlb_run_phases", "vlb_read_fields",
           "vlb_write_fields", "vlb_line_length", "vlb_destroy", "vlb_last_error", "vlb_set_timing",
           "vlb_lbm_timing", "vlb_biot_savart_scratch_bytes", "vlb_biot_savart", "vlb_set_graphs", "vlb_set_overlap",
           "vlb_biot_savart_noalloc", "vlb_step_async", "vlb_query", "vlb_query_stats", "vlb_channel_bytes",
           "vlb_kernel_timing"]
BUSY = 1
ASYNC_DEPTH = 4  # vlb_step_async calls a channel holds in flight
TIMED_LBM, TIMED_BIOT_SAVART = 0, 1  # kernel kinds of the event-timed mode


class Params(C.Structure):
    _fields_ = [
        ("n", C.c_int32 * 3), ("wall", C.c_int32 * 3), ("stream_axis", C.c_int32),
        ("vfm_substeps", C.c_int32), ("couple", C.c_int32), ("force_form", C.c_int32),
        ("max_points", C.c_int32), ("storage", C.c_int32), ("wall_images", C.c_int32), ("reserved", C.c_int32),
        ("tau", C.c_double), ("rho0", C.c_double), ("body_force", C.c_double * 3),
        ("heater_vn", C.c_double), ("pin_vn", C.c_double), ("init_vn", C.c_double * 3),
        ("kappa", C.c_double), ("alpha", C.c_double), ("alpha_p", C.c_double),
        ("rho_s_over_rho_n", C.c_double), ("core_a", C.c_double),
        ("dxi_min", C.c_double), ("dxi_max", C.c_double),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class VlbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libvlb {ERR.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libvlb.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libvlb.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)
        L.vlb_create_channel.argtypes = [C.POINTER(Params), C.POINTER(Allocator), vp, C.POINTER(vp)]
        L.vlb_seed_vortices.argtypes = [vp, dp, ip, C.c_int32]
        L.vlb_step.argtypes = [vp, C.c_int32]
        L.vlb_run_phases.argtypes = [vp, C.c_int32]
        L.vlb_read_fields.argtypes = [vp, C.c_int32, vp, C.c_size_t, C.POINTER(C.c_size_t)]
        L.vlb_write_fields.argtypes = [vp, C.c_int32, vp, C.c_size_t]
        L.vlb_line_length.argtypes = [vp, dp]
        L.vlb_destroy.argtypes = [vp]
        L.vlb_destroy.restype = None
        L.vlb_last_error.argtypes = []
        L.vlb_last_error.restype = C.c_char_p
        L.vlb_set_timing.argtypes = [vp, C.c_int32]
        L.vlb_set_graphs.argtypes = [vp, C.c_int32]
        L.vlb_set_overlap.argtypes = [vp, C.c_int32]
        L.vlb_lbm_timing.argtypes = [vp, dp, C.POINTER(C.c_int64)]
        L.vlb_kernel_timing.argtypes = [vp, C.c_int32, dp, C.POINTER(C.c_int64)]
        L.vlb_biot_savart_scratch_bytes.argtypes = [C.c_int32]
        L.vlb_biot_savart_scratch_bytes.restype = C.c_size_t
        L.vlb_biot_savart.argtypes = [C.POINTER(Params), vp, vp, C.c_int32, vp, vp, C.c_size_t, vp]
        L.vlb_biot_savart_noalloc.argtypes = [C.POINTER(Params), vp, vp, C.c_int32, vp, vp]
        L.vlb_step_async.argtypes = [vp, C.c_int32]
        L.vlb_query.argtypes = [vp]
        L.vlb_query_stats.argtypes = [vp, C.POINTER(C.c_double)]
        L.vlb_channel_bytes.argtypes = [C.POINTER(Params)]
        L.vlb_channel_bytes.restype = C.c_size_t
        _lib = L
    return _lib


def check(rc: int):
    if rc != OK:
        raise VlbError(rc, lib().vlb_last_error().decode())


def make_params(d: dict) -> Params:
    p = Params()
    names = {f[0] for f in Params._fields_}
    for k, v in d.items():
        if k not in names:
            continue
        if isinstance(v, (list, tuple)):
            getattr(p, k)[:] = list(v)
        else:
            setattr(p, k, v)
    return p


class TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the C ABI."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self._alloc = ALLOC_FN(self._a)
        self._free = FREE_FN(self._f)
        self.struct = Allocator(None, self._alloc, self._free)

    def _a(self, ctx, nbytes, stream):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0)
        except Exception:
            return None

    def _f(self, ctx, ptr, stream):
        self.torch.cuda.caching_allocator_delete(ptr)


class Channel:
    """A lattice + filament set resident on the GPU (see include/vlb.h)."""

    def __init__(self, params: dict, stream=None, torch_alloc: bool = True, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libvlb needs a CUDA device")
        torch.cuda.set_device(device)
        self.params = dict(params)
        self._p = make_params(params)
        # a created stream by default: the step can then be replayed as a CUDA graph
        self.stream = stream if stream is not None else torch.cuda.Stream(device)
        self._alloc = TorchAllocator(device) if torch_alloc else None
        h = C.c_void_p()
        check(lib().vlb_create_channel(C.byref(self._p), C.byref(self._alloc.struct) if self._alloc else None,
                                       C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.n = tuple(int(v) for v in params["n"])
        self.ncell = self.n[0] * self.n[1] * self.n[2]

    def close(self):
        if getattr(self, "h", None):
            lib().vlb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def seed(self, xyz, nxt):
        xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
        nxt = np.ascontiguousarray(nxt, np.int32)
        check(lib().vlb_seed_vortices(self.h, xyz.ctypes.data_as(C.POINTER(C.c_double)),
                                      nxt.ctypes.data_as(C.POINTER(C.c_int32)), len(nxt)))

    def step(self, nsteps: int = 1, raise_on_error: bool = True) -> int:
        rc = lib().vlb_step(self.h, nsteps)
        if raise_on_error:
            check(rc)
        return rc

    def step_async(self, nsteps: int):
        """Queue nsteps coupled steps on the channel's stream and return."""
        check(lib().vlb_step_async(self.h, nsteps))

    def query(self) -> bool:
        """True once the oldest queued call has finished (raises on a device error)."""
        rc = lib().vlb_query(self.h)
        if rc == BUSY:
            return False
        check(rc)
        return True

    def query_stats(self) -> np.ndarray:
        """STATS record of the queued call that query() completed last."""
        out = np.zeros(16)
        check(lib().vlb_query_stats(self.h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def run_phases(self, mask: int, raise_on_error: bool = True) -> int:
        rc = lib().vlb_run_phases(self.h, mask)
        if raise_on_error:
            check(rc)
        return rc

    def stats(self) -> np.ndarray:
        out = np.zeros(16)
        written = C.c_size_t()
        check(lib().vlb_read_fields(self.h, FIELD_STATS, out.ctypes.data_as(C.c_void_p), out.nbytes,
                                    C.byref(written)))
        return out

    def n_points(self) -> int:
        return int(self.stats()[0])

    def read(self, which: int) -> np.ndarray:
        N = self.n_points() if which in (FIELD_POS, FIELD_VEL, FIELD_NEXT) else None
        shapes = {
            FIELD_RHO: ((self.ncell,), np.float32), FIELD_U: ((3, self.ncell), np.float32),
            FIELD_FSTAR: ((19, self.ncell), np.float32), FIELD_FDEV: ((19, self.ncell), np.float32),
            FIELD_FORCE: ((3, self.ncell), np.float32),
            FIELD_POS: ((N, 3), np.float64), FIELD_VEL: ((N, 3), np.float64), FIELD_NEXT: ((N,), np.int32),
            FIELD_PLANE_VS: ((self.n[2],), np.float64), FIELD_STATS: ((16,), np.float64),
            FIELD_LINE_PROFILE: ((self.n[2],), np.float64),
        }
        shape, dt = shapes[which]
        out = np.zeros(shape, dt)
        written = C.c_size_t()
        check(lib().vlb_read_fields(self.h, which, out.ctypes.data_as(C.c_void_p), out.nbytes, C.byref(written)))
        return out

    def write(self, which: int, arr):
        arr = np.ascontiguousarray(arr, np.float32)
        check(lib().vlb_write_fields(self.h, which, arr.ctypes.data_as(C.c_void_p), arr.nbytes))

    def line_length(self) -> float:
        out = C.c_double()
        check(lib().vlb_line_length(self.h, C.byref(out)))
        return out.value

    def set_graphs(self, enable: bool):
        check(lib().vlb_set_graphs(self.h, 1 if enable else 0))

    def set_overlap(self, enable: bool):
        check(lib().vlb_set_overlap(self.h, 1 if enable else 0))

    def set_timing(self, enable: bool):
        check(lib().vlb_set_timing(self.h, 1 if enable else 0))

    def lbm_timing(self):
        return self.kernel_timing(TIMED_LBM)

    def kernel_timing(self, kind: int):
        """(total ms, launches) of one kernel kind since set_timing(True)."""
        ms, n = C.c_double(), C.c_int64()
        check(lib().vlb_kernel_timing(self.h, kind, C.byref(ms), C.byref(n)))
        return ms.value, n.value


def biot_savart(params: dict, pos_dev: int, next_dev: int, n: int, vel_dev: int, scratch_dev: int,
                scratch_bytes: int, stream: int):
    """Stand-alone nonlocal Biot-Savart velocity (device pointers as ints)."""
    p = make_params(params)
    check(lib().vlb_biot_savart(C.byref(p), C.c_void_p(pos_dev), C.c_void_p(next_dev), n, C.c_void_p(vel_dev),
                                C.c_void_p(scratch_dev), scratch_bytes, C.c_void_p(stream)))


def biot_savart_scratch_bytes(n: int) -> int:
    return int(lib().vlb_biot_savart_scratch_bytes(n))


def biot_savart_noalloc(params: dict, pos_dev: int, next_dev: int, n: int, vel_dev: int, stream: int):
    """Allocation-free stand-alone Biot-Savart velocity (device pointers as
    ints; at most 65536 points; calls on overlapping streams race)."""
    p = make_params(params)
    check(lib().vlb_biot_savart_noalloc(C.byref(p), C.c_void_p(pos_dev), C.c_void_p(next_dev), n,
                                        C.c_void_p(vel_dev), C.c_void_p(stream)))


def channel_bytes(params: dict) -> int:
    """Device bytes a channel with these parameters allocates (0 if invalid)."""
    return int(lib().vlb_channel_bytes(C.byref(make_params(params))))
