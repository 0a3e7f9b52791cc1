"""GB300-native sparse exact Gaussian processes (arXiv 2205.09070).

The compute path is the CUDA library libgpsparse (csrc/, C ABI in
include/gpsparse.h); this package holds its build script, a thin ctypes
binding, a torch.autograd wrapper and the seeded synthetic workload
generators.
"""

from .gpsparse import (GP, GP_FP32_MIXED, GP_FP64, GPError, default_opts, load,  # noqa: F401
                       status_string)
