"""GB300-native multigrid GPW (FFTDF) collocation / integration path.

The compute path is libgpw (CUDA for sm_103a + cuFFT), reached through the C ABI in
``include/gpw.h``; :mod:`.binding` marshals torch tensors into it.
"""
from .binding import Plan, Batch, GpwError, load, lib_path  # noqa: F401

__all__ = ["Plan", "Batch", "GpwError", "load", "lib_path"]
