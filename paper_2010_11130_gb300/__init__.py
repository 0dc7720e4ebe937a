"""GB300 l-AIR algebraic multigrid + GMRES for space-time HDG trace systems.

The compute path is libair.so (hand-written CUDA for sm_103a, C ABI in
include/air.h); this package holds its sources, the in-tree build and the
ctypes binding.
"""
from .air import (CSR, AirError, Hierarchy, default_options, gmres_solve, lib, setup,  # noqa: F401
                  spmv, status_string, kernel_launches)
from .build import build  # noqa: F401
