"""Seeded space-time HDG input generator (mesh, assembly, condensation, scaling).

Shared by the CPU oracle tests and the GPU path as the source of the trace
systems they solve.  It holds none of the AIR / GMRES arithmetic.
"""
from .assemble import Problem, TraceSystem, assemble, l2_error, reconstruct, trace_full  # noqa: F401
from .mesh import build_mesh, choose_reflection  # noqa: F401
from . import problems  # noqa: F401
