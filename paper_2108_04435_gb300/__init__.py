"""GB300-native coupled vortex-filament / lattice-Boltzmann step (arXiv 2108.04435).

The compute path lives in ``libvlb.so`` (hand-written CUDA for sm_103a behind a
C ABI, declared in ``include/vlb.h``).  ``vlb`` is the thin ctypes binding;
``inputs`` holds the seeded synthetic input generators and ``configs`` the
workload presets.  Importing this package loads nothing; the binding loads the
CUDA library on first use and raises if it has not been built.
"""
__all__ = ["vlb", "inputs", "configs", "build"]
