"""GB300-native matrix-free unfitted DG Poisson operator (arXiv 2404.07911).

The compute path is libunfitted.so (C ABI in include/unfitted.h, CUDA kernels for sm_103a);
this package holds its build script and a thin ctypes binding.  There is no CPU fallback:
importing works without a GPU, but applying an operator needs the CUDA library and a device.
"""
from .binding import (UF_FP32, UF_FP64, UnfittedError, UnfittedOperator, debug_fail_allocation,  # noqa: F401
                      debug_live_allocations, load_library)
