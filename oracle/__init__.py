"""CPU oracle of the AIR-preconditioned GMRES path -- test infrastructure only.

Python marshalling around the plain C oracle in air_oracle.c (see that file
for the method and every reading of the paper it takes).  Only the tests, the
package smoke check and the benchmark's CPU baseline import this module; the
product path never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "air_oracle.c")
_LIB = os.path.join(_HERE, "_air_oracle.so")
_lib = None

I64P = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
I32P = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
F64P = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FP contraction) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    lib.ora_spmv.argtypes = [C.c_int64, I64P, I32P, F64P, F64P, F64P]
    lib.ora_spmv.restype = None
    lib.ora_setup.argtypes = [C.c_int64, I64P, I32P, F64P, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                              C.c_int, C.c_char_p, C.c_double, C.c_int64, C.POINTER(C.c_int)]
    lib.ora_hash_frac.argtypes = [C.c_uint64]
    lib.ora_hash_frac.restype = C.c_double
    lib.ora_setup.restype = C.c_void_p
    lib.ora_free.argtypes = [C.c_void_p]
    lib.ora_nlevels.argtypes = [C.c_void_p]
    lib.ora_nlevels.restype = C.c_int
    lib.ora_level_info.argtypes = [C.c_void_p, C.c_int, I64P]
    lib.ora_level_copy.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    lib.ora_level_copy.restype = C.c_int
    lib.ora_vcycle.argtypes = [C.c_void_p, F64P, F64P]
    lib.ora_gmres.argtypes = [C.c_int64, I64P, I32P, F64P, C.c_void_p, F64P, F64P, C.c_double,
                              C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p]
    lib.ora_gmres.restype = C.c_int
    lib.ora_bicgstab.argtypes = [C.c_int64, I64P, I32P, F64P, C.c_void_p, F64P, F64P, C.c_double, C.c_int,
                                 C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.ora_bicgstab.restype = C.c_int
    _lib = lib
    return lib


def _csr(row_ptr, col, val):
    return (np.ascontiguousarray(row_ptr, dtype=np.int64), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


def spmv(row_ptr, col, val, x) -> np.ndarray:
    """y = A x, row by row."""
    rp, ci, v = _csr(row_ptr, col, val)
    n = len(rp) - 1
    y = np.empty(n)
    _load().ora_spmv(n, rp, ci, v, np.ascontiguousarray(x, dtype=np.float64), y)
    return y


@dataclass
class Level:
    n: int
    A: tuple                # (row_ptr, col, val)
    S: tuple = None         # (row_ptr, col) strength pattern
    cf: np.ndarray = None   # int8, 1 = C
    cid: np.ndarray = None  # int32, coarse id or -1
    R: tuple = None         # (row_ptr, col, val), nc rows
    pcol: np.ndarray = None
    pw: np.ndarray = None
    nc: int = 0
    n_singular: int = 0
    max_m: int = 0


class Hierarchy:
    """Oracle AIR hierarchy; owns the C object."""

    def __init__(self, handle, lib, copy_levels=True):
        self._h, self._lib = handle, lib
        self.levels = []
        for l in range(lib.ora_nlevels(handle) if copy_levels else 0):
            info = np.zeros(8, dtype=np.int64)
            lib.ora_level_info(handle, l, info)
            n, nnz, snnz, nc, rnnz, nsing, maxm = (int(t) for t in info[:7])
            A = (self._get(l, 0, n + 1, np.int64), self._get(l, 1, nnz, np.int32), self._get(l, 2, nnz, np.float64))
            L = Level(n=n, A=A, nc=nc, n_singular=nsing, max_m=maxm)
            if nc > 0:
                L.S = (self._get(l, 3, n + 1, np.int64), self._get(l, 4, snnz, np.int32))
                L.cf = self._get(l, 5, n, np.int8)
                L.cid = self._get(l, 6, n, np.int32)
                L.R = (self._get(l, 7, nc + 1, np.int64), self._get(l, 8, rnnz, np.int32),
                       self._get(l, 9, rnnz, np.float64))
                L.pcol = self._get(l, 10, n, np.int32)
                L.pw = self._get(l, 11, n, np.float64)
            self.levels.append(L)

    def sizes(self):
        """(rows, stored entries) of every level, without copying the arrays."""
        out = []
        for l in range(self._lib.ora_nlevels(self._h)):
            info = np.zeros(8, dtype=np.int64)
            self._lib.ora_level_info(self._h, l, info)
            out.append((int(info[0]), int(info[1])))
        return out

    def _get(self, l, what, count, dtype):
        out = np.empty(count, dtype=dtype)
        if count and self._lib.ora_level_copy(self._h, l, what, out.ctypes.data_as(C.c_void_p)) != 0:
            raise RuntimeError("oracle level array missing")
        return out

    def vcycle(self, b) -> np.ndarray:
        """One V-cycle x = M^{-1} b from a zero initial guess."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        self._lib.ora_vcycle(self._h, b, x)
        return x

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.ora_free(self._h)
            self._h = None


class OracleError(RuntimeError):
    pass


def setup(row_ptr, col, val, theta=0.25, distance=1, max_coarse=1000, max_levels=25,
          max_dense=4096, relax="FCF", omega=1.0, theta_r=None, copy_levels=True,
          falgout_block=0) -> Hierarchy:
    """Build the AIR hierarchy (strength, RS splitting, l-AIR R, one-point P, RAP).

    theta is the strength threshold of the C/F splitting and one-point P;
    theta_r (default: theta) that of the l-AIR neighbourhoods of R.  With
    copy_levels=False the level arrays stay inside the C object (levels is
    empty; vcycle and gmres still work), which saves the copy on large runs.
    falgout_block > 0 replaces the first pass by the Falgout-style splitting
    with index blocks of that many points (see air_oracle.c)."""
    lib = _load()
    rp, ci, v = _csr(row_ptr, col, val)
    st = C.c_int(0)
    h = lib.ora_setup(len(rp) - 1, rp, ci, v, float(theta), float(theta if theta_r is None else theta_r),
                      int(distance), int(max_coarse),
                      int(max_levels), int(max_dense), relax.encode(), float(omega), int(falgout_block),
                      C.byref(st))
    if not h:
        raise OracleError(f"oracle setup failed with status {st.value}")
    H = Hierarchy(h, lib, copy_levels)
    if st.value != 0:
        raise OracleError(f"oracle setup failed with status {st.value}")
    return H


def gmres(row_ptr, col, val, H, b, rtol=1e-8, restart=30, max_iter=1000):
    """Right-preconditioned flexible GMRES(restart) with MGS; x0 = 0.

    Returns (x, iters, relres, converged, history of relative residual estimates).
    """
    lib = _load()
    rp, ci, v = _csr(row_ptr, col, val)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    it, rr = C.c_int(0), C.c_double(0.0)
    hist = np.zeros(max_iter + 1)
    rc = lib.ora_gmres(len(rp) - 1, rp, ci, v, H._h if H is not None else None, b, x, float(rtol),
                       int(restart), int(max_iter), C.byref(it), C.byref(rr),
                       hist.ctypes.data_as(C.c_void_p))
    return x, it.value, rr.value, rc == 0, hist[: it.value + 1]


def bicgstab(row_ptr, col, val, H, b, rtol=1e-12, max_iter=1000):
    """Right-preconditioned BiCGSTAB with one V-cycle of H as M^{-1} (identity if H is None).

    Returns (x, iterations, true relative residual, converged)."""
    lib = _load()
    rp, ci, v = _csr(row_ptr, col, val)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    it = C.c_int(0)
    rr = C.c_double(0.0)
    rc = lib.ora_bicgstab(len(rp) - 1, rp, ci, v, H._h if H is not None else None, b, x, float(rtol),
                          int(max_iter), C.byref(it), C.byref(rr))
    return x, it.value, rr.value, rc == 0



def hash_frac(x: int) -> float:
    """The oracle's SplitMix64 fraction of x (for pins of the Falgout-style splitting)."""
    return _load().ora_hash_frac(int(x))
