"""Space-time HDG assembly, static condensation and block scaling.

Builds the statically condensed trace system S Lambda = H of the space-time
HDG method (Section 2.3, eqs. st-hdg and bilin; Section 2.5, eqs. linsys and
systemLambda), then scales it on the left by the inverse of its facet
block diagonal (Section 4, solver settings), giving the system
    A x = b,   A = D_b^{-1} S,   b = D_b^{-1} H
that the AIR-preconditioned GMRES path solves.

Terms of B_h((u, lambda), (v, mu)) per element K (test functions v, mu;
a_hat = (1, a), a_hat_n = n_t + a.n, spatial normal n, spatial gradient):
  volume      -u a_hat.grad_hat(v) + nu grad(u).grad(v)
  facet       sigma(u, lambda)(v - mu) - nu (u - lambda) grad(v).n
  sigma       1/2 (a_hat_n (u + lambda) + |a_hat_n| (u - lambda))      (upwind)
              - nu grad(u).n + nu alpha / h_K (u - lambda)             (eq. 7)
  Neumann     1/2 (a_hat_n + |a_hat_n|) lambda mu  on dE_N
with alpha = 10 p^2 and h_K the longest edge of K.  Right-hand side:
  (f, v)_K + (g_N, mu)_{dE_N}.
Dirichlet facets (the spatial boundary for all t) carry the L2 projection of
g_D and are removed from the unknowns.  Neumann facets are the t = t0 and
t = tN faces; their spatial normal is zero, so g_N = -zeta a_hat_n u there,
which imposes the initial condition at t0 and is zero at the outflow tN.

This module is the seeded input generator shared by the CPU oracle tests and
the GPU path; it contains none of the AIR / GMRES arithmetic.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from .mesh import DIRICHLET, NEUMANN, Mesh
from .reference import monomials, n_elem, n_trace, simplex_quadrature, trace_basis


class RefData:
    """Reference-element tables for degree p in D space-time dimensions."""

    def __init__(self, D: int, p: int, q: Optional[int] = None):
        self.D, self.p = D, p
        q = p + 2 if q is None else q
        self.xq, self.wq = simplex_quadrature(D, q)                 # volume rule
        self.phi, self.gphi = monomials(self.xq, p)                 # (nq, nb), (nq, nb, D)
        self.sq, self.wf = simplex_quadrature(D - 1, q)             # facet rule (canonical)
        self.psi = trace_basis(self.sq, p)                          # (nqf, b)
        self.nb, self.b = n_elem(D, p), n_trace(D, p)
        self.perms = list(itertools.permutations(range(D)))
        self.perm_index = {pm: i for i, pm in enumerate(self.perms)}
        # barycentric coordinates of the canonical facet points
        beta = np.concatenate([1.0 - self.sq.sum(-1, keepdims=True), self.sq], axis=-1)  # (nqf, D)
        ref_verts = np.concatenate([np.zeros((1, D)), np.eye(D)], axis=0)              # (D+1, D)
        nqf = self.sq.shape[0]
        self.xi_f = np.empty((D + 1, len(self.perms), nqf, D))
        for k in range(D + 1):
            loc = [j for j in range(D + 1) if j != k]
            for s, pm in enumerate(self.perms):
                vsel = ref_verts[[loc[pm[m]] for m in range(D)]]          # canonical order
                self.xi_f[k, s] = beta @ vsel
        self.phi_f, self.gphi_f = monomials(self.xi_f, p)    # (D+1, D!, nqf, nb[, D])
        # reference stiffness tensor T[k, l, i, j] = sum_q w_q d_k phi_i d_l phi_j
        self.T = np.einsum("q,qik,qjl->klij", self.wq, self.gphi, self.gphi)
        # grad of barycentric coordinates in reference coordinates
        self.gbary = np.concatenate([-np.ones((1, D)), np.eye(D)], axis=0)  # (D+1, D)


@dataclass
class Problem:
    """One space-time advection-diffusion problem on a Kuhn mesh."""
    D: int
    n: int
    p: int
    nu: float
    velocity: Callable[[np.ndarray], np.ndarray]     # (..., D) -> (..., D-1)
    source: Callable[[np.ndarray], np.ndarray]       # (..., D) -> (...)
    g_dirichlet: Callable[[np.ndarray], np.ndarray]  # (..., D) -> (...)
    u_initial: Callable[[np.ndarray], np.ndarray]    # (..., D) -> (...), used at t = t0
    exact: Optional[Callable[[np.ndarray], np.ndarray]] = None
    reflect: Optional[tuple] = None
    lower: Optional[tuple] = None
    upper: Optional[tuple] = None
    vertex_map: Optional[Callable[[np.ndarray], np.ndarray]] = None
    elem_velocity: Optional[np.ndarray] = None       # (E, D-1) piecewise-constant override
    alpha: Optional[float] = None
    name: str = ""
    spec: Optional[tuple] = None                     # (factory name, kwargs) to rebuild in a worker


@dataclass
class TraceSystem:
    """Block-scaled trace system A x = b in CSR (row_ptr int64, col int32, val f64)."""
    n: int
    b: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    rhs: np.ndarray
    free_facets: np.ndarray          # global facet id of each free facet (facet-major DOFs)
    lam_dirichlet: np.ndarray        # (F, b) trace values on Dirichlet facets
    mesh: Mesh = None
    local: Optional[tuple] = None    # (A^{-1}B, A^{-1}F) per element, for reconstruction
    S_diag: Optional[np.ndarray] = None  # (Ff, b, b) unscaled diagonal blocks (kept if asked)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def _geometry(mesh: Mesh, e: np.ndarray):
    X = mesh.verts[mesh.elems[e]]                     # (E, D+1, D)
    J = np.swapaxes(X[:, 1:, :] - X[:, :1, :], 1, 2)  # J[:, :, k] = X_{k+1} - X_0
    Jinv = np.linalg.inv(J)
    det = np.abs(np.linalg.det(J))
    D = mesh.D
    h = np.zeros(len(e))
    for i in range(D + 1):
        for j in range(i + 1, D + 1):
            h = np.maximum(h, np.linalg.norm(X[:, i] - X[:, j], axis=-1))
    return X, J, Jinv, det, h


def _element_velocity(prob: Problem, e: np.ndarray, x: np.ndarray) -> np.ndarray:
    if prob.elem_velocity is not None:
        v = prob.elem_velocity[e]
        return np.broadcast_to(v[:, None, :], x.shape[:2] + (v.shape[-1],))
    return prob.velocity(x)


def element_matrices(mesh: Mesh, prob: Problem, ref: RefData, e: np.ndarray):
    """Local HDG matrices of elements e: A (E,nb,nb), B (E,nb,nt), C (E,nt,nb),
    Dm (E,nt,nt), F (E,nb), G (E,nt) with nt = (D+1) b trace DOFs ordered by
    local facet k then canonical node m."""
    D, p, nu = mesh.D, prob.p, prob.nu
    alpha = 10.0 * p * p if prob.alpha is None else prob.alpha
    nb, b = ref.nb, ref.b
    nt = (D + 1) * b
    E = len(e)
    X, J, Jinv, det, h = _geometry(mesh, e)
    fact = math.factorial
    # ---- volume terms
    xq = X[:, None, 0, :] + np.einsum("edk,qk->eqd", J, ref.xq)      # (E, nq, D)
    W = det[:, None] * ref.wq[None, :]                                 # (E, nq)
    a = _element_velocity(prob, e, xq)
    ahat = np.concatenate([np.ones(xq.shape[:2] + (1,)), a], axis=-1)  # (E, nq, D)
    at = np.einsum("ekd,eqd->eqk", Jinv, ahat)                         # Jinv @ a_hat
    adv = np.einsum("eqk,qik->eqi", at, ref.gphi)                      # a_hat.grad_hat(phi_i)
    # A[i, j] += -int phi_j a_hat.grad_hat(phi_i)
    A = -np.einsum("eqi,eq,qj->eij", adv, W, ref.phi, optimize=True)
    if nu != 0.0:
        G_sp = np.swapaxes(Jinv, 1, 2)[:, 1:, :]                       # spatial rows of Jinv^T
        Mm = np.einsum("esk,esl->ekl", G_sp, G_sp)
        A += nu * det[:, None, None] * np.einsum("ekl,klij->eij", Mm, ref.T, optimize=True)
    Fv = np.einsum("eq,eq,qi->ei", W, prob.source(xq), ref.phi, optimize=True)

    B = np.zeros((E, nb, nt))
    C = np.zeros((E, nt, nb))
    Dm = np.zeros((E, nt, nt))
    Gv = np.zeros((E, nt))
    vol = det / fact(D)
    glob = mesh.elems[e]
    psi = ref.psi                                                      # (nqf, b)
    for k in range(D + 1):
        loc = [j for j in range(D + 1) if j != k]
        order = np.argsort(glob[:, loc], axis=1, kind="stable")        # canonical perm
        pidx = np.array([ref.perm_index[tuple(r)] for r in order.tolist()]) if E else np.zeros(0, int)
        phif = ref.phi_f[k][pidx]                                      # (E, nqf, nb)
        gphif = ref.gphi_f[k][pidx]                                    # (E, nqf, nb, D)
        xif = ref.xi_f[k][pidx]                                        # (E, nqf, D)
        xf = X[:, None, 0, :] + np.einsum("edk,eqk->eqd", J, xif)
        gl = np.einsum("ekd,k->ed", Jinv, ref.gbary[k])             # Jinv^T grad_ref lambda_k
        gnorm = np.linalg.norm(gl, axis=-1)
        nhat = -gl / gnorm[:, None]                                    # outward unit normal
        area = D * vol * gnorm
        Wf = area[:, None] * ref.wf[None, :] * fact(D - 1)             # (E, nqf)
        af = _element_velocity(prob, e, xf)
        an = nhat[:, None, 0] + np.einsum("eqd,ed->eq", af, nhat[:, 1:])
        cup = 0.5 * (an + np.abs(an))
        cdn = 0.5 * (an - np.abs(an))
        pen = (nu * alpha / h)[:, None]
        vsp = np.concatenate([np.zeros((E, 1)), nhat[:, 1:]], axis=-1)
        jv = np.einsum("ekd,ed->ek", Jinv, vsp)                        # grad(.).n = gref . (Jinv v)
        dn = np.einsum("eqik,ek->eqi", gphif, jv)                      # (E, nqf, nb)
        sl = slice(k * b, (k + 1) * b)
        # A: (cup + pen) u v - nu (grad u.n) v - nu u (grad v.n)
        A += np.einsum("eq,eqi,eqj->eij", Wf * (cup + pen), phif, phif, optimize=True)
        if nu != 0.0:
            t = np.einsum("eq,eqi,eqj->eij", Wf, phif, dn, optimize=True)   # t[i,j] = int phi_i dn_j
            A -= nu * (t + np.swapaxes(t, 1, 2))
        # B[i, m]: (cdn - pen) lambda v + nu lambda grad(v).n
        B[:, :, sl] = np.einsum("eq,eqi,qm->eim", Wf * (cdn - pen), phif, psi, optimize=True)
        if nu != 0.0:
            B[:, :, sl] += nu * np.einsum("eq,eqi,qm->eim", Wf, dn, psi, optimize=True)
        # C[m, j]: -(cup + pen) u mu + nu grad(u).n mu
        C[:, sl, :] = -np.einsum("eq,eqj,qm->emj", Wf * (cup + pen), phif, psi, optimize=True)
        if nu != 0.0:
            C[:, sl, :] += nu * np.einsum("eq,eqj,qm->emj", Wf, dn, psi, optimize=True)
        # D[m, l]: -(cdn - pen) lambda mu  (+ cup lambda mu on Neumann facets)
        fid = mesh.elem_facets[e, k]
        neu = (mesh.facet_kind[fid] == NEUMANN).astype(np.float64)[:, None]
        coef = -(cdn - pen) + neu * cup
        Dm[:, sl, sl] = np.einsum("eq,ql,qm->eml", Wf * coef, psi, psi, optimize=True)
        # G: g_N = -zeta a_hat_n u_initial on the Neumann facets (spatial normal is zero)
        if np.any(neu):
            gN = np.where(an < 0.0, -an * prob.u_initial(xf), 0.0) * neu
            Gv[:, sl] = np.einsum("eq,eq,qm->em", Wf, gN, psi, optimize=True)
    return A, B, C, Dm, Fv, Gv


def dirichlet_values(mesh: Mesh, prob: Problem, ref: RefData) -> np.ndarray:
    """L2 projection of g_D onto P_p of each Dirichlet facet (canonical frame)."""
    D, b = mesh.D, ref.b
    lam = np.zeros((mesh.n_facets, b))
    fids = np.nonzero(mesh.facet_kind == DIRICHLET)[0]
    if len(fids) == 0:
        return lam
    W = mesh.verts[mesh.facets[fids]]                                  # (Fd, D, D) canonical
    Tm = np.swapaxes(W[:, 1:, :] - W[:, :1, :], 1, 2)                  # (Fd, D, D-1)
    xf = W[:, None, 0, :] + np.einsum("edk,qk->eqd", Tm, ref.sq)
    # surface measure of the (D-1)-simplex: sqrt(det(T^T T)) / (D-1)!
    g = np.einsum("edk,edl->ekl", Tm, Tm)
    meas = np.sqrt(np.linalg.det(g)) / math.factorial(D - 1)
    Wf = meas[:, None] * ref.wf[None, :] * math.factorial(D - 1)
    M = np.einsum("eq,qm,ql->eml", Wf, ref.psi, ref.psi)
    r = np.einsum("eq,eq,qm->em", Wf, prob.g_dirichlet(xf), ref.psi)
    lam[fids] = np.linalg.solve(M, r[..., None])[..., 0]
    return lam


def _condense_chunk(mesh: Mesh, prob: Problem, ref: RefData, e: np.ndarray, keep_local: bool):
    A, B, C, Dm, Fv, Gv = element_matrices(mesh, prob, ref, e)
    rhs = np.concatenate([B, Fv[:, :, None]], axis=2)
    X = np.linalg.solve(A, rhs)                      # A^{-1} [B, F]
    S = Dm - C @ X[:, :, :-1]
    H = Gv - np.einsum("emi,ei->em", C, X[:, :, -1])
    nf, b = mesh.D + 1, ref.b
    SK = S.reshape(len(e), nf, b, nf, b).transpose(0, 1, 3, 2, 4)
    HK = H.reshape(len(e), nf, b)
    loc = (X[:, :, :-1], X[:, :, -1]) if keep_local else None
    return SK, HK, loc


_WORKER_STATE = {}


def _worker_chunk(spec, start, stop):
    """Process-pool task: rebuild the problem and mesh from spec (cached per
    worker), condense elements [start, stop)."""
    from . import problems
    from .mesh import build_mesh
    key = repr(spec)
    if _WORKER_STATE.get("key") != key:
        prob = problems.make(spec)
        mesh = build_mesh(prob.D, prob.n, reflect=prob.reflect, lower=prob.lower, upper=prob.upper,
                          vertex_map=prob.vertex_map)
        _WORKER_STATE.update(key=key, prob=prob, mesh=mesh, ref=RefData(prob.D, prob.p))
    st = _WORKER_STATE
    SK, HK, _ = _condense_chunk(st["mesh"], st["prob"], st["ref"], np.arange(start, stop), False)
    return start, stop, SK, HK


def assemble(prob: Problem, mesh: Optional[Mesh] = None, chunk: int = 16384,
             keep_local: bool = False, scale: bool = True, keep_diag: bool = False,
             workers: int = 1) -> TraceSystem:
    """Assemble, condense and block-scale; returns the trace system in CSR.

    Free facets keep the global (sorted-vertex) facet order; DOF = r*b + m for
    free facet r and canonical node m.  Within a row, columns ascend.  The
    diagonal block of the scaled matrix is the identity by construction and is
    stored as its b diagonal ones only (the roundoff-level entries of
    D_b^{-1} S_ff - I are dropped).  With scale=False the unscaled S is
    returned with its full diagonal blocks.
    """
    from .mesh import build_mesh
    if mesh is None:
        mesh = build_mesh(prob.D, prob.n, reflect=prob.reflect, lower=prob.lower,
                          upper=prob.upper, vertex_map=prob.vertex_map)
    D, p = mesh.D, prob.p
    ref = RefData(D, p)
    b = ref.b
    E, F = mesh.n_elems, mesh.n_facets
    nf = D + 1
    SK = np.empty((E, nf, nf, b, b))
    HK = np.empty((E, nf, b))
    local = (np.empty((E, ref.nb, nf * b)), np.empty((E, ref.nb))) if keep_local else None
    if workers > 1 and prob.spec is not None and not keep_local and prob.elem_velocity is None:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        bounds = [(s0, min(E, s0 + chunk)) for s0 in range(0, E, chunk)]
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            futs = [ex.submit(_worker_chunk, prob.spec, a, z) for a, z in bounds]
            for f in futs:
                a, z, SKc, HKc = f.result()
                SK[a:z] = SKc
                HK[a:z] = HKc
    else:
        for s0 in range(0, E, chunk):
            e = np.arange(s0, min(E, s0 + chunk))
            SKc, HKc, loc = _condense_chunk(mesh, prob, ref, e, keep_local)
            SK[e] = SKc
            HK[e] = HKc
            if keep_local:
                local[0][e] = loc[0]
                local[1][e] = loc[1]
    lamD = dirichlet_values(mesh, prob, ref)

    kind = mesh.facet_kind
    free = kind != DIRICHLET
    free_ids = np.nonzero(free)[0]
    Ff = len(free_ids)
    rnum = -np.ones(F, dtype=np.int64)
    rnum[free_ids] = np.arange(Ff)

    # diagonal blocks and rhs, summed over the (<= 2) adjacent elements in element order
    fe, fl = mesh.facet_elems, mesh.facet_local
    Sd = SK[fe[:, 0], fl[:, 0], fl[:, 0]].copy()
    Hf = HK[fe[:, 0], fl[:, 0]].copy()
    two = fe[:, 1] >= 0
    Sd[two] += SK[fe[two, 1], fl[two, 1], fl[two, 1]]
    Hf[two] += HK[fe[two, 1], fl[two, 1]]

    # off-diagonal blocks (f, g): exactly one element holds both facets
    kk, ll = np.nonzero(~np.eye(nf, dtype=bool))
    fa = mesh.elem_facets[:, kk].reshape(-1)                 # (E*12,)
    ga = mesh.elem_facets[:, ll].reshape(-1)
    blk = SK[:, kk, ll].reshape(-1, b, b)
    # move Dirichlet columns to the rhs of free rows
    dcol = ~free[ga] & free[fa]
    if np.any(dcol):
        contrib = np.einsum("kij,kj->ki", blk[dcol], lamD[ga[dcol]])
        np.subtract.at(Hf, fa[dcol], contrib)
    keep = free[fa] & free[ga]
    fa, ga, blk = rnum[fa[keep]], rnum[ga[keep]], blk[keep]
    Sd, Hf = Sd[free_ids], Hf[free_ids]

    if scale:
        Dinv = np.linalg.inv(Sd)
        blk = Dinv[fa] @ blk
        rhs = np.einsum("fij,fj->fi", Dinv, Hf).reshape(-1)
    else:
        rhs = Hf.reshape(-1)

    order = np.lexsort((ga, fa))
    fa, ga, blk = fa[order], ga[order], blk[order]
    nblk = np.bincount(fa, minlength=Ff)                     # off-diagonal blocks per facet row
    bstart = np.concatenate([[0], np.cumsum(nblk)[:-1]])
    rank = np.arange(len(fa)) - bstart[fa]                   # rank within its block row
    n_before = np.bincount(fa, weights=(ga < fa), minlength=Ff).astype(np.int64)

    dlen = 1 if scale else b
    rowlen = np.repeat(nblk * b + dlen, b)                   # same for all b rows of a facet
    N = Ff * b
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(rowlen, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    ii = np.arange(b)
    # off-diagonal entries: row (f, i), position rank*b + j (+ dlen if g > f)
    rows = fa[:, None] * b + ii[None, :]                                 # (nb, b)
    base = row_ptr[rows] + (rank * b + dlen * (ga > fa))[:, None]        # (nb, b)
    pos = base[:, :, None] + ii[None, None, :]                           # (nb, b, b)
    col[pos.reshape(-1)] = (ga[:, None, None] * b + ii[None, None, :]).repeat(b, 1).reshape(-1).astype(np.int32)
    val[pos.reshape(-1)] = blk.reshape(-1)
    del pos, base
    # diagonal block
    f_all = np.arange(Ff)
    drow = f_all[:, None] * b + ii[None, :]                              # (Ff, b)
    dbase = row_ptr[drow] + (n_before * b)[:, None]
    if scale:
        col[dbase.reshape(-1)] = drow.reshape(-1).astype(np.int32)
        val[dbase.reshape(-1)] = 1.0
    else:
        dpos = dbase[:, :, None] + ii[None, None, :]
        col[dpos.reshape(-1)] = (f_all[:, None, None] * b + ii[None, None, :]).repeat(b, 1).reshape(-1).astype(np.int32)
        val[dpos.reshape(-1)] = Sd.reshape(-1)
    return TraceSystem(n=N, b=b, row_ptr=row_ptr, col=col, val=val, rhs=rhs,
                       free_facets=free_ids, lam_dirichlet=lamD, mesh=mesh, local=local,
                       S_diag=Sd if keep_diag else None)


def trace_full(system: TraceSystem, x: np.ndarray) -> np.ndarray:
    """All facet trace values (F, b): the solution on free facets, g_D on Dirichlet ones."""
    lam = system.lam_dirichlet.copy()
    lam[system.free_facets] = x.reshape(-1, system.b)
    return lam


def reconstruct(system: TraceSystem, x: np.ndarray) -> np.ndarray:
    """Element coefficients U = A^{-1}(F - B Lambda) (Section 2.5), (E, nb)."""
    if system.local is None:
        raise ValueError("assemble(..., keep_local=True) is required")
    lam = trace_full(system, x)
    Lk = lam[system.mesh.elem_facets].reshape(system.mesh.n_elems, -1)
    AinvB, AinvF = system.local
    return AinvF - np.einsum("eij,ej->ei", AinvB, Lk)


def l2_error(system: TraceSystem, prob: Problem, x: np.ndarray, chunk: int = 65536) -> float:
    """Space-time L2 error ||u - u_h|| over the mesh (Section 5.1) with the volume rule."""
    mesh = system.mesh
    ref = RefData(mesh.D, prob.p)
    U = reconstruct(system, x)
    tot = 0.0
    for s in range(0, mesh.n_elems, chunk):
        e = np.arange(s, min(mesh.n_elems, s + chunk))
        X, J, Jinv, det, h = _geometry(mesh, e)
        xq = X[:, None, 0, :] + np.einsum("edk,qk->eqd", J, ref.xq)
        uh = U[e] @ ref.phi.T
        tot += float(np.sum(det[:, None] * ref.wq[None, :] * (prob.exact(xq) - uh) ** 2))
    return math.sqrt(tot)
