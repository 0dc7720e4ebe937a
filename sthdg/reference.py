"""Reference-simplex tools for the space-time HDG input generator.

Quadrature, element bases and facet (trace) bases on the reference simplex
{xi >= 0, sum(xi) <= 1} in D = d+1 space-time dimensions (D = 2 for 1D+time,
D = 3 for 2D+time).  The element space is P_p(K) and the trace space is
P_p on each facet (Section 2.3, definitions of V_h and M_h).
"""
from __future__ import annotations

import itertools
import math
from functools import lru_cache

import numpy as np
from scipy.special import roots_jacobi


def multi_indices(dim: int, p: int) -> np.ndarray:
    """All exponent tuples alpha in N^dim with |alpha| <= p, lexicographic."""
    out = [a for a in itertools.product(range(p + 1), repeat=dim) if sum(a) <= p]
    return np.array(sorted(out), dtype=np.int64).reshape(-1, dim)


@lru_cache(maxsize=None)
def simplex_quadrature(dim: int, q: int):
    """Collapsed (Stroud conical product) Gauss-Jacobi rule on the reference simplex.

    Uses the Duffy map x_1 = u_1, x_2 = u_2 (1-u_1), x_3 = u_3 (1-u_1)(1-u_2),
    whose Jacobian (1-u_1)^(dim-1) (1-u_2)^(dim-2) ... is absorbed into the
    Gauss-Jacobi weights.  With q points per direction the rule integrates
    polynomials of total degree <= 2q-1 exactly.  Weights sum to 1/dim!.
    Returns (points (nq, dim), weights (nq,)).
    """
    if dim == 0:
        return np.zeros((1, 0)), np.ones(1)
    us, ws = [], []
    for k in range(dim):
        alpha = dim - 1 - k
        x, w = roots_jacobi(q, alpha, 0.0)
        us.append((1.0 + x) / 2.0)
        ws.append(w / 2.0 ** (alpha + 1))
    pts, wts = [], []
    for idx in itertools.product(range(q), repeat=dim):
        u = [us[k][idx[k]] for k in range(dim)]
        w = 1.0
        for k in range(dim):
            w *= ws[k][idx[k]]
        x = np.empty(dim)
        scale = 1.0
        for k in range(dim):
            x[k] = u[k] * scale
            scale *= 1.0 - u[k]
        pts.append(x)
        wts.append(w)
    return np.array(pts), np.array(wts)


def monomials(xi: np.ndarray, p: int):
    """Element basis: monomials xi^alpha, |alpha| <= p, and their reference gradients.

    The Schur complement S = D - C A^{-1} B does not depend on the choice of
    element basis, so the simplest complete basis of P_p is used.
    xi: (..., dim).  Returns values (..., nb) and gradients (..., nb, dim).
    """
    dim = xi.shape[-1]
    alphas = multi_indices(dim, p)
    nb = len(alphas)
    val = np.ones(xi.shape[:-1] + (nb,))
    grad = np.zeros(xi.shape[:-1] + (nb, dim))
    for b, al in enumerate(alphas):
        for k in range(dim):
            val[..., b] *= xi[..., k] ** al[k]
        for d in range(dim):
            if al[d] == 0:
                continue
            g = np.full(xi.shape[:-1], float(al[d]))
            for k in range(dim):
                e = al[k] - (1 if k == d else 0)
                g = g * xi[..., k] ** e
            grad[..., b, d] = g
    return val, grad


@lru_cache(maxsize=None)
def lattice(dim: int, p: int) -> np.ndarray:
    """Equispaced nodes beta/p, |beta| <= p, of the reference dim-simplex, lexicographic."""
    return multi_indices(dim, p).astype(np.float64) / max(p, 1)


@lru_cache(maxsize=None)
def _lagrange_coeffs(dim: int, p: int) -> np.ndarray:
    nodes = lattice(dim, p)
    V, _ = monomials(nodes, p)            # V[i, b] = m_b(node_i)
    return np.linalg.inv(V)               # L_j = sum_b C[b, j] m_b


def trace_basis(s: np.ndarray, p: int) -> np.ndarray:
    """Lagrange basis of P_p on the reference (D-1)-simplex at points s (..., D-1).

    Node j is the j-th lattice point in lexicographic order; basis j is 1 at
    node j and 0 at the others.  Returns (..., b) with b = C(p+D-1, D-1).
    """
    dim = s.shape[-1]
    m, _ = monomials(s, p)
    return m @ _lagrange_coeffs(dim, p)


def n_trace(D: int, p: int) -> int:
    """Trace DOFs per facet: dim P_p on a (D-1)-simplex."""
    return math.comb(p + D - 1, D - 1)


def n_elem(D: int, p: int) -> int:
    """Element DOFs: dim P_p on a D-simplex."""
    return math.comb(p + D, D)
