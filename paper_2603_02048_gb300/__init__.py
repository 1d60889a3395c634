"""GB300 (sm_103a) curved-ray heat-haze engine.

The hot path of arXiv 2603.02048 Sec. 3.3 -- particle splat, Gladstone-Dale
refractive-index volume, adaptive curved-ray march and background lookup --
as CUDA kernels behind the C ABI of include/hh.h. ``hh`` is the ctypes
binding (same names as the C functions); ``build`` compiles libhh.so.
"""
from . import hh  # noqa: F401

__all__ = ["hh"]
