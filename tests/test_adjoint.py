"""The adjoint of the condensed solve, pinned on the CPU.

u = A^{-1} b for the block-scaled trace system (Section 2.5).  For a loss
L(u) the gradient is dL/db = lambda with A^T lambda = dL/du, and dL/da_ij =
-lambda_i u_j on the stored entries.  These tests pin that formula against
central finite differences with dense solves, and check that the oracle's
l-AIR setup and GMRES also solve the transposed (reversed-flow) system.
"""
import numpy as np
import scipy.sparse as sp

import oracle
from sthdg import assemble
from sthdg.problems import manufactured_2d


def _dense(s, val=None):
    v = s.val if val is None else val
    return sp.csr_matrix((v, s.col, s.row_ptr), shape=(s.n, s.n)).toarray()


def _loss(A, b, ut):
    u = np.linalg.solve(A, b)
    return 0.5 * float(np.sum((u - ut) ** 2))


def test_dense_adjoint_gradient_matches_central_differences():
    s = assemble(manufactured_2d(2, 1, 1e-2))
    rng = np.random.default_rng(11)
    A = _dense(s)
    b = s.rhs.copy()
    ut = rng.standard_normal(s.n)
    u = np.linalg.solve(A, b)
    lam = np.linalg.solve(A.T, u - ut)
    h = 1e-6
    for k in rng.choice(s.n, 4, replace=False):
        e = np.zeros(s.n)
        e[k] = h
        fd = (_loss(A, b + e, ut) - _loss(A, b - e, ut)) / (2 * h)
        assert abs(fd - lam[k]) <= 1e-6 * max(1.0, abs(lam[k]))
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    gval = -lam[rows] * u[s.col]
    for e in rng.choice(len(s.val), 4, replace=False):
        vp, vm = s.val.copy(), s.val.copy()
        vp[e] += h
        vm[e] -= h
        fd = (_loss(_dense(s, vp), b, ut) - _loss(_dense(s, vm), b, ut)) / (2 * h)
        assert abs(fd - gval[e]) <= 1e-6 * max(1.0, abs(gval[e]))


def test_transpose_keeps_unit_diagonal():
    # block scaling makes every diagonal entry of A exactly 1; A^T inherits it
    s = assemble(manufactured_2d(3, 2, 1e-6))
    At = sp.csr_matrix((s.val, s.col, s.row_ptr), shape=(s.n, s.n)).T.tocsr()
    assert np.array_equal(At.diagonal(), np.ones(s.n))


def test_oracle_solves_the_transposed_system():
    s = assemble(manufactured_2d(6, 2, 1e-6))
    At = sp.csr_matrix((s.val, s.col, s.row_ptr), shape=(s.n, s.n)).T.tocsr()
    At.sort_indices()
    rp, ci, v = At.indptr.astype(np.int64), At.indices.astype(np.int32), At.data
    g = np.random.default_rng(3).standard_normal(s.n)
    Ht = oracle.setup(rp, ci, v, theta=0.25, max_coarse=100)
    lam, it_t, rr, ok, _ = oracle.gmres(rp, ci, v, Ht, g, rtol=1e-8)
    assert ok and rr <= 1e-8
    assert np.linalg.norm(g - At @ lam) <= 1e-8 * np.linalg.norm(g) * (1 + 1e-6)
    # the reversed flow is coarsened as well as the forward one
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    _, it_f, _, ok_f, _ = oracle.gmres(s.row_ptr, s.col, s.val, H, s.rhs, rtol=1e-8)
    assert ok_f and it_t <= 2 * it_f + 5


def test_mapped_noisy_recipe():
    """Time-dependent mapped domain with noisy element velocities: the map
    keeps the space-time cube's boundary, the velocities are (1, 0.5) plus
    0.1 N(0,1) from default_rng(4) in element order, and block scaling still
    gives a unit diagonal."""
    from sthdg.mesh import build_mesh
    from sthdg.problems import mapped_noisy
    pr = mapped_noisy(3, 1, 1e-4)
    m0 = build_mesh(3, 3, reflect=pr.reflect)
    m1 = build_mesh(3, 3, reflect=pr.reflect, vertex_map=pr.vertex_map)
    V0, V1 = m0.verts, m1.verts
    on_bnd = np.any((V0[:, 1:] == 0.0) | (V0[:, 1:] == 1.0), axis=1) | (V0[:, 0] == 0.0) | (V0[:, 0] == 1.0)
    assert np.allclose(V1[on_bnd], V0[on_bnd], atol=1e-15)
    assert np.abs(V1 - V0).max() > 1e-3
    rng = np.random.default_rng(4)
    assert np.array_equal(pr.elem_velocity, np.array([1.0, 0.5]) + 0.1 * rng.standard_normal((m0.n_elems, 2)))
    s = assemble(pr)
    A = sp.csr_matrix((s.val, s.col, s.row_ptr), shape=(s.n, s.n))
    assert np.array_equal(A.diagonal(), np.ones(s.n))


def test_mapped_noisy_adjoint_matches_central_differences():
    from sthdg.problems import mapped_noisy
    s = assemble(mapped_noisy(2, 1, 1e-4))
    rng = np.random.default_rng(12)
    A = _dense(s)
    ut = rng.standard_normal(s.n)
    u = np.linalg.solve(A, s.rhs)
    lam = np.linalg.solve(A.T, u - ut)
    h = 1e-6
    for k in rng.choice(s.n, 3, replace=False):
        e = np.zeros(s.n)
        e[k] = h
        fd = (_loss(A, s.rhs + e, ut) - _loss(A, s.rhs - e, ut)) / (2 * h)
        assert abs(fd - lam[k]) <= 1e-6 * max(1.0, abs(lam[k]))
