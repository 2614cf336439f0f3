"""GB300-native explicit Runge-Kutta-Chebyshev solver for nonlinear EQS fields.

The compute path is the CUDA library ``_lib/libeqs.so`` (C ABI in
include/eqs.h); ``eqs`` is its ctypes binding.  Build with ``build.build()``.
"""
from . import build  # noqa: F401
