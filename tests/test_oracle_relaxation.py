"""Pins of the oracle's relaxation sweeps (Section 4 solver settings: the paper
post-relaxes with forward Gauss-Seidel, first on the F points and then on all
points; the library's default is FCF-Jacobi).

The V-cycle operator is composed densely from the level matrices by the
textbook matrix form of each sweep over a point set S:
  Jacobi        x <- x + omega D_SS^{-1} (b - A x)_S
  Gauss-Seidel  x <- x + (D_SS / omega + L_SS)^{-1} (b - A x)_S
with L_SS the strictly lower (by index) part of A restricted to S, and
compared with the oracle's point-by-point sweeps.  A lower-triangular system
is solved exactly by one forward Gauss-Seidel sweep over all points, so one
V-cycle with that relaxation must return A^{-1} b.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from sthdg import assemble
from sthdg.problems import manufactured_1d, manufactured_2d


def _sp(rp, ci, v, shape):
    return sp.csr_matrix((v, ci, rp), shape=shape)


def _dense_vcycle(H, relax, omega):
    def level_op(l):
        L = H.levels[l]
        A = _sp(*L.A, (L.n, L.n)).toarray()
        if l == len(H.levels) - 1:
            return np.linalg.inv(A)
        R = _sp(*L.R, (L.nc, L.n)).toarray()
        P = np.zeros((L.n, H.levels[l + 1].n))
        rows = np.nonzero(L.pcol >= 0)[0]
        P[rows, L.pcol[rows]] = L.pw[rows]
        M = P @ level_op(l + 1) @ R
        I = np.eye(L.n)
        for c in relax:
            if c in "Aa":
                S = np.arange(L.n)
            else:
                S = np.nonzero(L.cf == (1 if c in "Cc" else 0))[0]
            ASS = A[np.ix_(S, S)]
            if c.isupper():
                B = np.diag(omega / np.diag(ASS))
            else:
                B = np.linalg.inv(np.diag(np.diag(ASS)) / omega + np.tril(ASS, -1))
            E = I[:, S]
            M = M + E @ B @ E.T @ (I - A @ M)
        return M
    return level_op(0)


@pytest.mark.parametrize("relax,omega", [("fa", 1.0), ("FCF", 1.0), ("fcf", 0.8), ("A", 0.7), ("Ff", 1.0)])
def test_vcycle_sweeps_equal_dense_composition(relax, omega):
    s = assemble(manufactured_1d(8, 1, 1e-3))
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=20, relax=relax, omega=omega)
    assert len(H.levels) >= 3
    Minv = _dense_vcycle(H, relax, omega)
    rng = np.random.default_rng(2)
    for _ in range(3):
        b = rng.standard_normal(s.n)
        want = Minv @ b
        assert np.allclose(H.vcycle(b), want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


def test_gauss_seidel_all_points_solves_lower_triangular_in_one_vcycle():
    """A unit lower-triangular (upwind) system: the forward sweep over all
    points is a forward substitution, so x = A^{-1} b whatever the coarse-grid
    correction left (Section 3.3: the ordered block Gauss-Seidel inverts the
    advective part exactly when the matrix graph is acyclic)."""
    rng = np.random.default_rng(5)
    n = 400
    M = np.eye(n)
    for i in range(1, n):
        for j in rng.choice(i, size=min(i, 3), replace=False):
            M[i, j] = -rng.uniform(0.2, 1.0)
    S = sp.csr_matrix(M)
    S.sort_indices()
    rp, ci, v = S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data
    H = oracle.setup(rp, ci, v, theta=0.25, max_coarse=20, relax="a")
    assert len(H.levels) >= 2
    b = rng.standard_normal(n)
    x = H.vcycle(b)
    assert np.linalg.norm(M @ x - b) <= 1e-12 * np.linalg.norm(b)
    # Jacobi over all points is not exact on the same system
    Hj = oracle.setup(rp, ci, v, theta=0.25, max_coarse=20, relax="A")
    assert np.linalg.norm(M @ Hj.vcycle(b) - b) > 1e-6 * np.linalg.norm(b)


def test_gauss_seidel_gmres_converges_on_trace_system():
    s = assemble(manufactured_2d(4, 1, 1e-4))
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100, relax="fa")
    x, it, rr, ok, _ = oracle.gmres(s.row_ptr, s.col, s.val, H, s.rhs, rtol=1e-10)
    A = _sp(s.row_ptr, s.col, s.val, (s.n, s.n))
    assert ok and np.linalg.norm(s.rhs - A @ x) <= 1e-10 * np.linalg.norm(s.rhs) * 1.0001
