"""GB300 l-AIR algebraic multigrid + GMRES for space-time HDG trace systems.

The compute path is libair.so (hand-written CUDA for sm_103a, C ABI in
include/air.h); this package holds its sources, the in-tree build and the
ctypes binding.
"""
from .air import (CSR, AdjointSolver, AirError, Hierarchy, bicgstab_solve, bicgstab_solve_multi,  # noqa: F401
                  csr_outer, default_options, vcycle_multi,
                  gmres_solve, gmres_solve_batch, kernel_launches, lib, setup, setup_batch, spmv,
                  status_string, transpose, transpose_scaled, block_diag_apply)
from .build import build  # noqa: F401
