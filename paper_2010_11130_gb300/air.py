"""Thin ctypes binding of libair.so (include/air.h).

Argument marshalling only: every step of setup, V-cycle and GMRES runs in the
library's CUDA kernels.  torch tensors provide device memory and streams.
The library must have been built (paper_2010_11130_gb300.build.build());
loading fails loudly if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from .build import LIB

AIR_OK = 0
AIR_NOT_CONVERGED = 1
AIR_PREC_F64 = 0
AIR_PREC_F32 = 1
AIR_PREC_BF16 = 2

EXPORTED = ["air_default_options", "air_setup", "air_vcycle", "air_spmv", "air_gmres_solve",
            "air_hierarchy_levels", "air_hierarchy_info", "air_hierarchy_export", "air_free",
            "air_status_string", "air_kernel_launches", "air_gmres_solve_noalloc", "air_setup_timings",
            "air_csr_transpose", "air_csr_outer", "air_setup_batch", "air_gmres_solve_batch",
            "air_bicgstab_solve", "air_vcycle_multi", "air_bicgstab_solve_multi",
            "air_vcycle_multi_f32", "air_hdg_points", "air_hdg_size", "air_hdg_assemble",
            "air_hdg_velocity_gradient", "air_csr_transpose_scaled", "air_block_diag_apply",
            "air_hierarchy_spmv"]


class air_csr(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("on_device", C.c_int)]


class air_options(C.Structure):
    _fields_ = [("theta", C.c_double), ("distance", C.c_int), ("relax", C.c_char * 16),
                ("omega", C.c_double), ("max_coarse", C.c_int), ("max_levels", C.c_int),
                ("max_dense", C.c_int), ("precision", C.c_int), ("restart", C.c_int),
                ("max_iter", C.c_int), ("validate", C.c_int), ("theta_r", C.c_double),
                ("falgout_block", C.c_int), ("block_size", C.c_int), ("autotune", C.c_int)]


class air_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("vcycles", C.c_int),
                ("status", C.c_int), ("relres", C.c_double)]


class air_level_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("nnz_s", C.c_int64), ("nc", C.c_int64),
                ("nnz_r", C.c_int64), ("n_singular", C.c_int64), ("max_m", C.c_int32),
                ("coarsest", C.c_int32), ("block_size", C.c_int32), ("lanes_f", C.c_int32),
                ("lanes_c", C.c_int32), ("lanes_r", C.c_int32)]


class air_hdg_mesh(C.Structure):
    _fields_ = [("D", C.c_int), ("n_verts", C.c_int64), ("n_elems", C.c_int64), ("n_facets", C.c_int64),
                ("verts", C.c_void_p), ("elems", C.c_void_p), ("elem_facets", C.c_void_p), ("facets", C.c_void_p),
                ("facet_elems", C.c_void_p), ("facet_kind", C.c_void_p)]


class air_hdg_ref(C.Structure):
    _fields_ = [("p", C.c_int), ("nb", C.c_int), ("b", C.c_int), ("nq", C.c_int), ("nqf", C.c_int),
                ("nperm", C.c_int), ("wq", C.c_void_p), ("xq", C.c_void_p), ("phi", C.c_void_p),
                ("gphi", C.c_void_p), ("wf", C.c_void_p), ("sq", C.c_void_p), ("psi", C.c_void_p),
                ("xi_f", C.c_void_p), ("phi_f", C.c_void_p), ("gphi_f", C.c_void_p), ("perms", C.c_void_p),
                ("dir_proj", C.c_void_p)]


class air_hdg_data(C.Structure):
    _fields_ = [("nu", C.c_double), ("alpha", C.c_double), ("vel_vol", C.c_void_p), ("src", C.c_void_p),
                ("vel_face", C.c_void_p), ("u0_face", C.c_void_p), ("g_dir", C.c_void_p)]


class AirError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else status_string(status))


_lib = None


def lib() -> C.CDLL:
    """Load libair.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"libair.so not built at {LIB}: run paper_2010_11130_gb300.build.build()")
    L = C.CDLL(LIB)
    L.air_default_options.argtypes = [C.POINTER(air_options)]
    L.air_default_options.restype = None
    L.air_setup.argtypes = [C.POINTER(air_csr), C.c_double, C.c_int, C.POINTER(air_options), C.c_void_p,
                            C.POINTER(C.c_void_p)]
    L.air_setup.restype = C.c_int
    L.air_vcycle.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.air_vcycle.restype = C.c_int
    L.air_spmv.argtypes = [C.POINTER(air_csr), C.c_void_p, C.c_void_p, C.c_void_p]
    L.air_spmv.restype = C.c_int
    L.air_hierarchy_spmv.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.air_hierarchy_spmv.restype = C.c_int
    L.air_gmres_solve.argtypes = [C.POINTER(air_csr), C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                  C.c_void_p, C.POINTER(air_solve_info)]
    L.air_gmres_solve.restype = C.c_int
    L.air_gmres_solve_noalloc.argtypes = [C.POINTER(air_csr), C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_double, C.c_void_p, C.POINTER(air_solve_info)]
    L.air_gmres_solve_noalloc.restype = C.c_int
    L.air_setup_timings.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.c_int]
    L.air_setup_timings.restype = C.c_int
    L.air_hierarchy_levels.argtypes = [C.c_void_p]
    L.air_hierarchy_levels.restype = C.c_int
    L.air_hierarchy_info.argtypes = [C.c_void_p, C.c_int, C.POINTER(air_level_info)]
    L.air_hierarchy_info.restype = C.c_int
    L.air_hierarchy_export.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    L.air_hierarchy_export.restype = C.c_int
    L.air_free.argtypes = [C.c_void_p]
    L.air_free.restype = None
    L.air_kernel_launches.argtypes = []
    L.air_kernel_launches.restype = C.c_ulonglong
    L.air_status_string.argtypes = [C.c_int]
    L.air_status_string.restype = C.c_char_p
    L.air_csr_transpose.argtypes = [C.POINTER(air_csr), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.air_csr_transpose.restype = C.c_int
    L.air_csr_outer.argtypes = [C.POINTER(air_csr), C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
    L.air_csr_outer.restype = C.c_int
    L.air_bicgstab_solve.argtypes = [C.POINTER(air_csr), C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                     C.c_void_p, C.POINTER(air_solve_info)]
    L.air_bicgstab_solve.restype = C.c_int
    L.air_vcycle_multi.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    L.air_vcycle_multi.restype = C.c_int
    L.air_vcycle_multi_f32.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    L.air_vcycle_multi_f32.restype = C.c_int
    L.air_bicgstab_solve_multi.argtypes = [C.POINTER(air_csr), C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                           C.c_double, C.c_void_p, C.POINTER(air_solve_info)]
    L.air_bicgstab_solve_multi.restype = C.c_int
    L.air_setup_batch.argtypes = [C.c_int, C.POINTER(air_csr), C.c_double, C.c_int, C.POINTER(air_options),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_int)]
    L.air_setup_batch.restype = C.c_int
    L.air_gmres_solve_batch.argtypes = [C.c_int, C.POINTER(air_csr), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_void_p), C.c_double, C.POINTER(C.c_void_p),
                                        C.POINTER(air_solve_info), C.POINTER(C.c_int)]
    L.air_gmres_solve_batch.restype = C.c_int
    L.air_csr_transpose_scaled.argtypes = [C.POINTER(air_csr), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p]
    L.air_csr_transpose_scaled.restype = C.c_int
    L.air_block_diag_apply.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    L.air_block_diag_apply.restype = C.c_int
    L.air_hdg_points.argtypes = [C.POINTER(air_hdg_mesh), C.POINTER(air_hdg_ref), C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
    L.air_hdg_points.restype = C.c_int
    L.air_hdg_size.argtypes = [C.POINTER(air_hdg_mesh), C.POINTER(air_hdg_ref), C.c_int, C.POINTER(C.c_int64),
                               C.POINTER(C.c_int64), C.c_void_p]
    L.air_hdg_size.restype = C.c_int
    L.air_hdg_assemble.argtypes = [C.POINTER(air_hdg_mesh), C.POINTER(air_hdg_ref), C.POINTER(air_hdg_data), C.c_int,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]
    L.air_hdg_assemble.restype = C.c_int
    L.air_hdg_velocity_gradient.argtypes = [C.POINTER(air_hdg_mesh), C.POINTER(air_hdg_ref), C.POINTER(air_hdg_data),
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.air_hdg_velocity_gradient.restype = C.c_int
    _lib = L
    return L


def status_string(st: int) -> str:
    return lib().air_status_string(int(st)).decode()


def kernel_launches() -> int:
    """Kernels libair has launched in this process (diagnostic counter)."""
    return int(lib().air_kernel_launches())


def _check(st: int, what: str):
    if st < 0:
        raise AirError(st, what)
    return st


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


@dataclass
class CSR:
    """CSR operand; arrays are torch tensors (device) or numpy arrays (host)."""
    row_ptr: object
    col: object
    val: object
    n: int

    @staticmethod
    def from_host(row_ptr, col, val, device="cuda"):
        import torch
        rp = torch.as_tensor(np.ascontiguousarray(row_ptr, dtype=np.int64)).to(device)
        ci = torch.as_tensor(np.ascontiguousarray(col, dtype=np.int32)).to(device)
        v = torch.as_tensor(np.ascontiguousarray(val, dtype=np.float64)).to(device)
        return CSR(rp, ci, v, len(row_ptr) - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def c(self) -> air_csr:
        on_dev = not isinstance(self.val, np.ndarray)
        ptr = (lambda t: t.data_ptr()) if on_dev else (lambda a: a.ctypes.data)
        return air_csr(self.n, self.n, self.nnz, ptr(self.row_ptr), ptr(self.col), ptr(self.val),
                       1 if on_dev else 0)


def default_options(**kw) -> air_options:
    o = air_options()
    lib().air_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "relax":
            v = v.encode()
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Hierarchy:
    """Library-owned AIR hierarchy (opaque pointer)."""

    _EXPORT = {"A.row_ptr": (0, np.int64), "A.col": (1, np.int32), "A.val": (2, np.float64),
               "S.row_ptr": (3, np.int64), "S.col": (4, np.int32), "cf": (5, np.int8),
               "cid": (6, np.int32), "R.row_ptr": (7, np.int64), "R.col": (8, np.int32),
               "R.val": (9, np.float64), "pcol": (10, np.int32)}

    def __init__(self, handle: int, A: CSR, precision: int):
        self._h = C.c_void_p(handle)
        self.A = A                      # keeps an aliased finest matrix alive
        self.precision = precision

    @property
    def handle(self):
        return self._h

    PHASES = ("strength", "transpose", "splitting", "lair", "onepoint_P", "rap", "coarsest", "other",
              "split_picks", "split_refills", "split_lines_searched")

    def setup_timings(self) -> dict:
        """Device milliseconds per setup phase (summed over levels)."""
        buf = (C.c_double * 11)()
        _check(lib().air_setup_timings(self._h, buf, 11), "air_setup_timings")
        return {k: float(buf[i]) for i, k in enumerate(self.PHASES)}

    def levels(self) -> int:
        return lib().air_hierarchy_levels(self._h)

    def info(self, level: int) -> air_level_info:
        inf = air_level_info()
        _check(lib().air_hierarchy_info(self._h, level, C.byref(inf)), "air_hierarchy_info")
        return inf

    def export(self, level: int, what: str) -> np.ndarray:
        inf = self.info(level)
        code, dt = self._EXPORT[what]
        size = {0: inf.n + 1, 1: inf.nnz, 2: inf.nnz, 3: inf.n + 1, 4: inf.nnz_s, 5: inf.n, 6: inf.n,
                7: inf.nc + 1, 8: inf.nnz_r, 9: inf.nnz_r, 10: inf.n}[code]
        out = np.empty(size, dtype=dt)
        if size:
            _check(lib().air_hierarchy_export(self._h, level, code, out.ctypes.data_as(C.c_void_p)),
                   f"air_hierarchy_export({what})")
        return out

    def spmv(self, x, y=None, stream=None):
        """air_hierarchy_spmv: y = A x with the FP64 copy of A the Krylov solves use."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(lib().air_hierarchy_spmv(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                        C.c_void_p(_stream(stream))), "air_hierarchy_spmv")
        return y

    def vcycle(self, b, x=None, stream=None):
        import torch
        if x is None:
            x = torch.empty_like(b)
        _check(lib().air_vcycle(self._h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                C.c_void_p(_stream(stream))), "air_vcycle")
        return x

    def free(self):
        if self._h is not None and self._h.value:
            lib().air_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def setup(A: CSR, theta: float = 0.25, distance: int = 1, stream=None, **opts) -> Hierarchy:
    """air_setup: build the l-AIR hierarchy of A on the GPU."""
    o = default_options(**opts)
    h = C.c_void_p(0)
    Ac = A.c()
    st = lib().air_setup(C.byref(Ac), float(theta), int(distance), C.byref(o),
                         C.c_void_p(_stream(stream) if Ac.on_device else 0), C.byref(h))
    _check(st, "air_setup")
    return Hierarchy(h.value, A, o.precision)


def spmv(A: CSR, x, y=None, stream=None):
    import torch
    if y is None:
        y = torch.empty_like(x)
    Ac = A.c()
    _check(lib().air_spmv(C.byref(Ac), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                          C.c_void_p(_stream(stream))), "air_spmv")
    return y


def gmres_solve(A: CSR, H: Hierarchy, b, x=None, rtol: float = 1e-8, stream=None):
    """air_gmres_solve.  Device tensors for device A; numpy arrays for host A."""
    Ac = A.c()
    inf = air_solve_info()
    if Ac.on_device:
        import torch
        if x is None:
            x = torch.empty_like(b)
        bp, xp, sp = b.data_ptr(), x.data_ptr(), _stream(stream)
    else:
        if x is None:
            x = np.empty_like(b)
        bp, xp, sp = b.ctypes.data, x.ctypes.data, 0
    st = lib().air_gmres_solve(C.byref(Ac), H.handle, C.c_void_p(bp), C.c_void_p(xp), float(rtol),
                               C.c_void_p(sp), C.byref(inf))
    _check(st, "air_gmres_solve")
    return x, inf


def bicgstab_solve(A: CSR, H: Hierarchy, b, x=None, rtol: float = 1e-12, stream=None):
    """air_bicgstab_solve.  Device tensors for device A; numpy arrays for host A."""
    Ac = A.c()
    inf = air_solve_info()
    if Ac.on_device:
        import torch
        if x is None:
            x = torch.empty_like(b)
        bp, xp, sp = b.data_ptr(), x.data_ptr(), _stream(stream)
    else:
        if x is None:
            x = np.empty_like(b)
        bp, xp, sp = b.ctypes.data, x.ctypes.data, 0
    st = lib().air_bicgstab_solve(C.byref(Ac), H.handle, C.c_void_p(bp), C.c_void_p(xp), float(rtol),
                                  C.c_void_p(sp), C.byref(inf))
    _check(st, "air_bicgstab_solve")
    return x, inf


def gmres_solve_noalloc(A: CSR, H: Hierarchy, b, x, rtol: float = 1e-8, stream=None):
    """air_gmres_solve_noalloc: the same solve with no device allocation.

    For callers whose device memory is fully pre-assigned (a pool or budget)
    or whose framework forbids allocation inside the solve phase.  A, b and x
    are device tensors; x must be preallocated by the caller.  The Krylov
    workspace is a fixed 32 MiB device array shared by all calls, so calls
    that overlap on the GPU race.
    """
    Ac = A.c()
    inf = air_solve_info()
    st = lib().air_gmres_solve_noalloc(C.byref(Ac), H.handle, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                       float(rtol), C.c_void_p(_stream(stream)), C.byref(inf))
    _check(st, "air_gmres_solve_noalloc")
    return x, inf


# ------------------------------------------------------------------ adjoint
def transpose(A: CSR, stream=None) -> CSR:
    """air_csr_transpose: A^T of a square device CSR, columns ascending, values bit for bit."""
    import torch
    dev = A.val.device
    rp = torch.empty(A.n + 1, dtype=torch.int64, device=dev)
    ci = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)[:A.nnz]
    v = torch.empty(max(A.nnz, 1), dtype=torch.float64, device=dev)[:A.nnz]
    Ac = A.c()
    _check(lib().air_csr_transpose(C.byref(Ac), C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()),
                                   C.c_void_p(v.data_ptr()), C.c_void_p(_stream(stream))), "air_csr_transpose")
    return CSR(rp, ci, v, A.n)


def transpose_scaled(A: CSR, b: int, diag, stream=None) -> CSR:
    """air_csr_transpose_scaled: D_b^{-T} A^T D_b^T for the block-scaled A = D_b^{-1} S
    (diag: the (n/b, b, b) device blocks D_b)."""
    import torch
    dev = A.val.device
    rp = torch.empty(A.n + 1, dtype=torch.int64, device=dev)
    ci = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)[:A.nnz]
    v = torch.empty(max(A.nnz, 1), dtype=torch.float64, device=dev)[:A.nnz]
    Ac = A.c()
    _check(lib().air_csr_transpose_scaled(C.byref(Ac), int(b), C.c_void_p(diag.data_ptr()), C.c_void_p(rp.data_ptr()),
                                          C.c_void_p(ci.data_ptr()), C.c_void_p(v.data_ptr()),
                                          C.c_void_p(_stream(stream))), "air_csr_transpose_scaled")
    return CSR(rp, ci, v, A.n)


def block_diag_apply(b: int, diag, op: int, x, y=None, stream=None):
    """air_block_diag_apply: y_k = op(D_k) x_k (op 0 D, 1 D^T, 2 D^{-1}, 3 D^{-T})."""
    import torch
    if y is None:
        y = torch.empty_like(x)
    _check(lib().air_block_diag_apply(int(x.shape[0]) // int(b), int(b), C.c_void_p(diag.data_ptr()), int(op),
                                      C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), C.c_void_p(_stream(stream))),
           "air_block_diag_apply")
    return y


def csr_outer(A: CSR, u, w, alpha: float = 1.0, out=None, stream=None):
    """air_csr_outer: out[e] = alpha * u[i] * w[j] over the stored entries (i, j) of A."""
    import torch
    if out is None:
        out = torch.empty(max(A.nnz, 1), dtype=torch.float64, device=A.val.device)[:A.nnz]
    Ac = A.c()
    _check(lib().air_csr_outer(C.byref(Ac), C.c_void_p(u.data_ptr()), C.c_void_p(w.data_ptr()), float(alpha),
                               C.c_void_p(out.data_ptr()), C.c_void_p(_stream(stream))), "air_csr_outer")
    return out


_SOLVE_FN = None


def _solve_fn():
    """torch.autograd.Function of u = A^{-1} b (built on first use)."""
    global _SOLVE_FN
    if _SOLVE_FN is None:
        import torch

        class AirSolve(torch.autograd.Function):
            @staticmethod
            def forward(ctx, b, val, solver):
                x, info = gmres_solve(solver.A, solver.H, b.detach().contiguous(), rtol=solver.rtol)
                solver.info = info
                if info.status != 0:
                    raise AirError(info.status, "forward solve did not converge")
                ctx.solver = solver
                ctx.save_for_backward(x)
                return x

            @staticmethod
            def backward(ctx, gx):
                (x,) = ctx.saved_tensors
                solver = ctx.solver
                lam = solver.solve_adjoint(gx.contiguous())
                gval = csr_outer(solver.A, lam, x, -1.0) if ctx.needs_input_grad[1] else None
                return lam, gval, None

        _SOLVE_FN = AirSolve
    return _SOLVE_FN


class AdjointSolver:
    """Forward and adjoint l-AIR solves of one matrix A, differentiable.

    solve(b) returns u = A^{-1} b as a torch tensor that autograd
    differentiates: the backward pass solves A^T lambda = dL/du with a second
    l-AIR hierarchy built on A^T (built on the first backward) and returns
    dL/db = lambda and, when A.val requires grad, dL/dA.val = -lambda_i u_j on
    the stored entries.  The hierarchies are built from A's values at
    construction time; rebuild the solver after changing them.
    """

    def __init__(self, A: CSR, rtol: float = 1e-8, theta: float = 0.25, block=None, **opts):
        """block = (b, diag): A is D_b^{-1} S with facet blocks of b unknowns and
        diag the (n/b, b, b) blocks D_b; the adjoint then solves the block-scaled
        similar matrix D_b^{-T} A^T D_b^T (identity diagonal blocks, like A)."""
        self.A, self.rtol, self.theta, self.opts = A, rtol, theta, opts
        self.block = block
        self.H = setup(A, theta=theta, **opts)
        self.At = self.Ht = None
        self.info = self.info_adjoint = None

    def adjoint_hierarchy(self):
        if self.Ht is None:
            self.At = transpose(self.A) if self.block is None else transpose_scaled(self.A, *self.block)
            self.Ht = setup(self.At, theta=self.theta, **self.opts)
        return self.At, self.Ht

    def solve_adjoint(self, g):
        At, Ht = self.adjoint_hierarchy()
        if self.block is not None:
            b, diag = self.block
            g = block_diag_apply(b, diag, 3, g)
        lam, info = gmres_solve(At, Ht, g, rtol=self.rtol)
        self.info_adjoint = info
        if info.status != 0:
            raise AirError(info.status, "adjoint solve did not converge")
        if self.block is not None:
            lam = block_diag_apply(b, diag, 1, lam)
        return lam

    def solve(self, b, val=None):
        return _solve_fn().apply(b, self.A.val if val is None else val, self)


# ------------------------------------------------------------------ batches
def setup_batch(As, theta: float = 0.25, distance: int = 1, streams=None, **opts):
    """air_setup_batch: independent setups at once, level by level, with each
    level's local l-AIR solves of all problems in one launch.

    Returns (hierarchies, statuses); a failed problem has hierarchy None.
    """
    k = len(As)
    o = default_options(**opts)
    arr = (air_csr * k)(*[A.c() for A in As])
    out = (C.c_void_p * k)()
    st = (C.c_int * k)()
    sp = None if streams is None else (C.c_void_p * k)(*[int(s.cuda_stream) for s in streams])
    lib().air_setup_batch(k, arr, float(theta), int(distance), C.byref(o), sp, out, st)
    hs = [Hierarchy(out[i], As[i], o.precision) if out[i] else None for i in range(k)]
    return hs, [int(x) for x in st]


def gmres_solve_batch(As, Hs, bs, xs=None, rtol: float = 1e-8, streams=None):
    """air_gmres_solve_batch: independent device solves in lockstep, the V-cycles of
    each round in one CUDA graph.  Returns (xs, infos, statuses)."""
    import torch
    k = len(As)
    if xs is None:
        xs = [torch.empty_like(b) for b in bs]
    arr = (air_csr * k)(*[A.c() for A in As])
    hp = (C.c_void_p * k)(*[H.handle.value for H in Hs])
    bp = (C.c_void_p * k)(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * k)(*[x.data_ptr() for x in xs])
    inf = (air_solve_info * k)()
    st = (C.c_int * k)()
    sp = None if streams is None else (C.c_void_p * k)(*[int(s.cuda_stream) for s in streams])
    r = lib().air_gmres_solve_batch(k, arr, hp, bp, xp, float(rtol), sp, inf, st)
    if r < 0 and all(int(x) >= 0 for x in st):
        _check(r, "air_gmres_solve_batch")
    return xs, [inf[i] for i in range(k)], [int(x) for x in st]


# ------------------------------------------------------- many right-hand sides
def vcycle_multi(H: Hierarchy, B, X=None, stream=None):
    """air_vcycle_multi (float64 B) or air_vcycle_multi_f32 (float32 B): X = M^{-1} B
    for an (n, k) row-major device tensor, k <= 32."""
    import torch
    if X is None:
        X = torch.empty_like(B)
    fn = lib().air_vcycle_multi_f32 if B.dtype == torch.float32 else lib().air_vcycle_multi
    _check(fn(H.handle, int(B.shape[1]), C.c_void_p(B.data_ptr()), C.c_void_p(X.data_ptr()),
              C.c_void_p(_stream(stream))), "air_vcycle_multi")
    return X


def bicgstab_solve_multi(A: CSR, H: Hierarchy, B, X=None, rtol: float = 1e-12, stream=None):
    """air_bicgstab_solve_multi on the columns of an (n, k) FP64 device tensor.  Returns (X, infos)."""
    import torch
    k = int(B.shape[1])
    if X is None:
        X = torch.empty_like(B)
    inf = (air_solve_info * k)()
    Ac = A.c()
    st = lib().air_bicgstab_solve_multi(C.byref(Ac), H.handle, k, C.c_void_p(B.data_ptr()),
                                        C.c_void_p(X.data_ptr()), float(rtol), C.c_void_p(_stream(stream)), inf)
    _check(st, "air_bicgstab_solve_multi")
    return X, [inf[j] for j in range(k)]
