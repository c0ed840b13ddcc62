"""GB300-native Hermite finite-difference residual and SSP-RK3 step (arXiv 2109.01286).

`hfd` is the Python binding of the C ABI declared in include/hfd.h; the computation runs in the
in-tree library `_lib/libhfd.so` (host C++ preprocessing + CUDA kernels for sm_103a), built by
`build.build()`.
"""
from . import hfd
from .hfd import Batch, HfdError, Mesh, Prep, measure_fma_peaks, options
from . import autograd

__all__ = ["hfd", "autograd", "Batch", "HfdError", "Mesh", "Prep", "measure_fma_peaks", "options"]
