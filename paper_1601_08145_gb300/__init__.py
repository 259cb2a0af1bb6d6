"""GB300 (sm_103a) implementation of one time step of the positivity-
preserving Lax-Wendroff DG method for the 2D Euler equations
(Moe, Rossmanith & Seal, arXiv:1601.08145).

The compute path is liblxw.so (CUDA kernels behind the C ABI of
include/lxw.h); :mod:`paper_1601_08145_gb300.lxw` is its ctypes binding.
"""
from . import lxw  # noqa: F401
