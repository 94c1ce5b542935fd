"""The CUDA library builds for sm_103a and exports every entry point that
include/vlb.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "vlb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vlb_[a-z_]+)\s*\(", txt)))


def test_library_exports_declared_symbols():
    from paper_2108_04435_gb300 import build, vlb
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(vlb.EXPORTS)


def test_binding_refuses_without_gpu():
    import torch
    from paper_2108_04435_gb300 import configs, vlb
    if torch.cuda.is_available():
        return
    p, _, _ = configs.config("ring32")
    try:
        vlb.Channel(p)
    except RuntimeError as e:
        assert "CUDA" in str(e)
    else:
        raise AssertionError("channel created without a GPU")


def test_standalone_scratch_fits_the_allocation_free_array():
    """The scratch size of the stand-alone Biot-Savart entry grows with n, so
    the allocation-free entry's fixed 19 MiB array, sized for its largest
    call (65536 points, include/vlb.h), holds every smaller call too."""
    from paper_2108_04435_gb300 import build
    lib = ctypes.CDLL(build.build())
    f = lib.vlb_biot_savart_scratch_bytes
    f.argtypes = [ctypes.c_int32]
    f.restype = ctypes.c_size_t
    ns = list(range(0, 65536, 37)) + [8191, 8192, 24575, 24576, 65535, 65536]
    sizes = [f(n) for n in sorted(ns)]
    assert all(a <= b for a, b in zip(sizes, sizes[1:]))
    assert all(s % 256 == 0 for s in sizes)
    assert f(65536) <= 19 << 20
    # at least the 80-byte source records of two slots per point
    assert f(65536) >= 80 * 2 * 65536
