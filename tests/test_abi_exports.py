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
