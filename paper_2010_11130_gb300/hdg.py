"""GPU assembly of the space-time HDG trace system (air_hdg_* in include/air.h).

Argument marshalling only: the quadrature-point coordinates, the element
matrices, the static condensation, the scatter into the facet CSR pattern,
the block scaling and the velocity gradient all run in libair's kernels.
The reference-element tables come from hdg_ref (computed once per (D, p) on
the host and copied to the device); the mesh arrays and the problem data
(velocity, source, initial and Dirichlet data at the quadrature points) are
the caller's input.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from .air import CSR, _check, _stream, air_hdg_data, air_hdg_mesh, air_hdg_ref, lib
from .hdg_ref import HdgReference


def _dev(a, dtype, device):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=dtype)).to(device)


class HdgTables:
    """Reference tables of (D, p) on the device."""

    def __init__(self, D: int, p: int, device="cuda"):
        import torch
        self.ref = HdgReference(D, p)
        r = self.ref
        self.D, self.p = D, p
        self._t = {}
        for name in ("wq", "xq", "phi", "gphi", "wf", "sq", "psi", "xi_f", "phi_f", "gphi_f", "dir_proj"):
            self._t[name] = _dev(getattr(r, name), np.float64, device)
        self._t["perms"] = _dev(r.perms, np.int32, device)
        self.c = air_hdg_ref(p, r.nb, r.b, r.nq, r.nqf, r.nperm,
                             *[self._t[k].data_ptr() for k in ("wq", "xq", "phi", "gphi", "wf", "sq", "psi",
                                                               "xi_f", "phi_f", "gphi_f", "perms", "dir_proj")])
        self.nq, self.nqf, self.b, self.nb = r.nq, r.nqf, r.b, r.nb
        del torch


class HdgMesh:
    """Mesh arrays on the device (int32 ids, float64 coordinates)."""

    def __init__(self, D, verts, elems, elem_facets, facets, facet_elems, facet_kind, device="cuda"):
        self.D = D
        self.verts = _dev(verts, np.float64, device)
        self.elems = _dev(elems, np.int32, device)
        self.elem_facets = _dev(elem_facets, np.int32, device)
        self.facets = _dev(facets, np.int32, device)
        self.facet_elems = _dev(facet_elems, np.int32, device)
        self.facet_kind = _dev(facet_kind, np.int8, device)
        self.n_verts, self.n_elems, self.n_facets = len(verts), len(elems), len(facets)
        self.c = air_hdg_mesh(D, self.n_verts, self.n_elems, self.n_facets, self.verts.data_ptr(),
                              self.elems.data_ptr(), self.elem_facets.data_ptr(), self.facets.data_ptr(),
                              self.facet_elems.data_ptr(), self.facet_kind.data_ptr())

    @staticmethod
    def from_mesh(m, device="cuda"):
        """From any object with the fields D, verts, elems, elem_facets, facets,
        facet_elems, facet_kind (e.g. the seeded Kuhn meshes of sthdg.mesh)."""
        return HdgMesh(m.D, m.verts, m.elems, m.elem_facets, m.facets, m.facet_elems, m.facet_kind, device)


def points(mesh: HdgMesh, tab: HdgTables, stream=None):
    """air_hdg_points: (x_vol (E, nq, D), x_face (E, D+1, nqf, D), x_facet (F, nqf, D))."""
    import torch
    dev = mesh.verts.device
    D = mesh.D
    xv = torch.empty((mesh.n_elems, tab.nq, D), dtype=torch.float64, device=dev)
    xf = torch.empty((mesh.n_elems, D + 1, tab.nqf, D), dtype=torch.float64, device=dev)
    xF = torch.empty((mesh.n_facets, tab.nqf, D), dtype=torch.float64, device=dev)
    _check(lib().air_hdg_points(C.byref(mesh.c), C.byref(tab.c), C.c_void_p(xv.data_ptr()),
                                C.c_void_p(xf.data_ptr()), C.c_void_p(xF.data_ptr()), C.c_void_p(_stream(stream))),
           "air_hdg_points")
    return xv, xf, xF


@dataclass
class HdgData:
    """Problem data at the quadrature points (device float64 tensors)."""
    nu: float
    alpha: float
    vel_vol: object           # (E, nq, D-1)
    vel_face: object          # (E, D+1, nqf, D-1)
    src: object = None        # (E, nq)
    u0_face: object = None    # (E, D+1, nqf)
    g_dir: object = None      # (F, nqf)

    def c(self):
        ptr = (lambda t: t.data_ptr() if t is not None else None)
        return air_hdg_data(self.nu, self.alpha, ptr(self.vel_vol), ptr(self.src), ptr(self.vel_face),
                            ptr(self.u0_face), ptr(self.g_dir))


@dataclass
class HdgSystem:
    A: CSR
    rhs: object               # (n,) device
    diag: object              # (n_free, b, b) unscaled diagonal blocks
    lam_dir: object           # (F, b) Dirichlet trace values
    scaled: bool


def assemble(mesh: HdgMesh, tab: HdgTables, data: HdgData, scale: bool = True, stream=None) -> HdgSystem:
    """air_hdg_size + air_hdg_assemble: the (block-scaled) trace system on the device."""
    import torch
    dev = mesh.verts.device
    n, nnz = C.c_int64(0), C.c_int64(0)
    sp = C.c_void_p(_stream(stream))
    _check(lib().air_hdg_size(C.byref(mesh.c), C.byref(tab.c), int(scale), C.byref(n), C.byref(nnz), sp),
           "air_hdg_size")
    n, nnz = n.value, nnz.value
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    ci = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)[:nnz]
    v = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)[:nnz]
    rhs = torch.empty(n, dtype=torch.float64, device=dev)
    diag = torch.empty((n // tab.b, tab.b, tab.b), dtype=torch.float64, device=dev)
    lam = torch.empty((mesh.n_facets, tab.b), dtype=torch.float64, device=dev)
    dc = data.c()
    _check(lib().air_hdg_assemble(C.byref(mesh.c), C.byref(tab.c), C.byref(dc), int(scale),
                                  C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()), C.c_void_p(v.data_ptr()),
                                  C.c_void_p(rhs.data_ptr()), C.c_void_p(diag.data_ptr()),
                                  C.c_void_p(lam.data_ptr()), sp), "air_hdg_assemble")
    return HdgSystem(CSR(rp, ci, v, n), rhs, diag, lam, bool(scale))


def velocity_gradient(mesh: HdgMesh, tab: HdgTables, data: HdgData, sys_: HdgSystem, lam, adj, stream=None):
    """air_hdg_velocity_gradient: dL/d(element velocity), (E, D-1), from the
    trace solution lam of the scaled system and its adjoint adj."""
    import torch
    grad = torch.empty((mesh.n_elems, mesh.D - 1), dtype=torch.float64, device=mesh.verts.device)
    dc = data.c()
    _check(lib().air_hdg_velocity_gradient(C.byref(mesh.c), C.byref(tab.c), C.byref(dc),
                                           C.c_void_p(sys_.diag.data_ptr()), C.c_void_p(sys_.lam_dir.data_ptr()),
                                           C.c_void_p(lam.data_ptr()), C.c_void_p(adj.data_ptr()),
                                           C.c_void_p(grad.data_ptr()), C.c_void_p(_stream(stream))),
           "air_hdg_velocity_gradient")
    return grad
