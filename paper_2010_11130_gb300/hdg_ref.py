"""Reference-element tables of the space-time HDG discretisation for the GPU
assembly (air_hdg_* in include/air.h).

The discretisation (Section 2.3: V_h = P_p per element, M_h = P_p per facet)
is fixed by three choices that the assembled trace system depends on, and
this module states them from their definitions:

* quadrature: the collapsed (conical-product) Gauss-Jacobi rule on the
  reference simplex with q = p + 2 points per direction.  Direction k of a
  dim-simplex uses the Jacobi weight (1 - x)^(dim-1-k) on [-1, 1]; its nodes
  and weights come from the eigen-decomposition of the Jacobi matrix of the
  three-term recurrence (Golub-Welsch).  The points are mapped by
  x_1 = u_1, x_2 = u_2 (1 - u_1), x_3 = u_3 (1 - u_1)(1 - u_2).
* trace basis: on each facet, the Lagrange basis of P_p at the equispaced
  lattice nodes beta / p (|beta| <= p, lexicographic order), in the facet's
  canonical frame, whose vertices are the facet's global vertex ids sorted
  ascending (both neighbours of a facet then agree on its basis).
* element basis: any basis of P_p gives the same Schur complement
  S = D - C A^{-1} B; monomials in the reference coordinates are used.

Everything here is per reference element (independent of the mesh size), and
is computed once on the host and copied to the device.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def gauss_jacobi(q: int, alpha: float):
    """Nodes and weights of the q-point Gauss rule on [-1, 1] for the weight
    (1 - x)^alpha (beta = 0), by Golub-Welsch."""
    a, bt = float(alpha), 0.0
    diag = np.empty(q)
    off = np.empty(max(q - 1, 0))
    diag[0] = (bt - a) / (a + bt + 2.0)
    for n in range(1, q):
        s = 2.0 * n + a + bt
        diag[n] = (bt * bt - a * a) / (s * (s + 2.0))
    for n in range(1, q):
        s = 2.0 * n + a + bt
        num = 4.0 * n * (n + a) * (n + bt) * (n + a + bt)
        off[n - 1] = math.sqrt(num / (s * s * (s + 1.0) * (s - 1.0)))
    J = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(J)
    mu0 = 2.0 ** (a + bt + 1.0) * math.gamma(a + 1.0) * math.gamma(bt + 1.0) / math.gamma(a + bt + 2.0)
    w = mu0 * V[0, :] ** 2
    return x, w


def simplex_rule(dim: int, q: int):
    """Collapsed Gauss-Jacobi rule on {xi >= 0, sum xi <= 1}: (points (nq, dim),
    weights (nq,)), exact for total degree 2q - 1; weights sum to 1/dim!."""
    if dim == 0:
        return np.zeros((1, 0)), np.ones(1)
    us, ws = [], []
    for k in range(dim):
        al = dim - 1 - k
        x, w = gauss_jacobi(q, al)
        us.append(0.5 * (x + 1.0))
        ws.append(w / 2.0 ** (al + 1))
    pts, wts = [], []
    for idx in itertools.product(range(q), repeat=dim):
        u = [us[k][idx[k]] for k in range(dim)]
        pt = np.empty(dim)
        fac = 1.0
        for k in range(dim):
            pt[k] = u[k] * fac
            fac *= 1.0 - u[k]
        pts.append(pt)
        wts.append(np.prod([ws[k][idx[k]] for k in range(dim)]))
    return np.array(pts), np.array(wts)


def exponents(dim: int, p: int):
    """Exponent tuples of P_p in dim variables, graded then lexicographic."""
    out = []
    for deg in range(p + 1):
        out += sorted(a for a in itertools.product(range(deg + 1), repeat=dim) if sum(a) == deg)
    return np.array(out, dtype=np.int64).reshape(-1, dim)


def monomial_table(pts: np.ndarray, p: int):
    """Values (n, nb) and reference gradients (n, nb, dim) of the monomials."""
    n, dim = pts.shape
    ex = exponents(dim, p)
    val = np.ones((n, len(ex)))
    grad = np.zeros((n, len(ex), dim))
    for j, a in enumerate(ex):
        for k in range(dim):
            val[:, j] *= pts[:, k] ** a[k]
        for d in range(dim):
            if a[d] == 0:
                continue
            g = np.full(n, float(a[d]))
            for k in range(dim):
                g *= pts[:, k] ** (a[k] - (1 if k == d else 0))
            grad[:, j, d] = g
    return val, grad


def lagrange_table(s: np.ndarray, p: int):
    """Lagrange basis of P_p on the (D-1)-simplex at points s (n, D-1): basis m
    is 1 at the m-th lattice node beta / p (|beta| <= p, lexicographic)."""
    dim = s.shape[1]
    nodes = np.array(sorted(a for a in itertools.product(range(p + 1), repeat=dim) if sum(a) <= p),
                     dtype=np.float64).reshape(-1, dim) / p
    Vn, _ = monomial_table(nodes, p)          # Vn[node, mono]
    Vs, _ = monomial_table(s, p)
    return Vs @ np.linalg.inv(Vn)             # (n, b): Vs @ C with Vn @ C = I


class HdgReference:
    """All reference tables for (D, p); arrays are float64 / int32 numpy."""

    def __init__(self, D: int, p: int):
        if D not in (2, 3) or p not in (1, 2, 3):
            raise ValueError("D in {2, 3} and p in {1, 2, 3}")
        self.D, self.p = D, p
        q = p + 2
        self.nb = math.comb(p + D, D)
        self.b = math.comb(p + D - 1, D - 1)
        self.xq, self.wq = simplex_rule(D, q)
        self.nq = len(self.wq)
        self.phi, self.gphi = monomial_table(self.xq, p)
        self.sq, self.wf = simplex_rule(D - 1, q)
        self.nqf = len(self.wf)
        self.psi = lagrange_table(self.sq, p)
        perms = list(itertools.permutations(range(D)))
        self.perms = np.array(perms, dtype=np.int32)
        self.nperm = len(perms)
        refv = np.vstack([np.zeros((1, D)), np.eye(D)])                  # reference vertices
        bary = np.hstack([1.0 - self.sq.sum(1, keepdims=True), self.sq])  # (nqf, D)
        self.xi_f = np.empty((D + 1, self.nperm, self.nqf, D))
        for k in range(D + 1):
            loc = [j for j in range(D + 1) if j != k]
            for s, pm in enumerate(perms):
                corners = refv[[loc[pm[m]] for m in range(D)]]             # canonical vertex m
                self.xi_f[k, s] = bary @ corners
        flat = self.xi_f.reshape(-1, D)
        v, g = monomial_table(flat, p)
        self.phi_f = v.reshape(D + 1, self.nperm, self.nqf, self.nb)
        self.gphi_f = g.reshape(D + 1, self.nperm, self.nqf, self.nb, D)
        # L2 projection onto the trace basis of one facet: lambda = P g(points)
        W = np.diag(self.wf)
        M = self.psi.T @ W @ self.psi
        self.dir_proj = np.linalg.solve(M, self.psi.T @ W)               # (b, nqf)

    def arrays(self):
        """The tables in the order of the air_hdg_ref structure."""
        return [self.xq, self.wq, self.phi, self.gphi, self.wf, self.sq, self.psi, self.xi_f, self.phi_f,
                self.gphi_f, self.perms, self.dir_proj]
