"""Pins of two oracle branches that the converged parity cases never reach.

* The restart of GMRES(m): once m inner steps are spent, the oracle solves
  H y = g, updates x <- x + Z y and starts a new Arnoldi cycle from the true
  residual b - A x (the Krylov outer loop; the paper names GMRES as the
  alternative to its BiCGSTAB in Section 5.1).  A small restart length forces
  several cycles, and an independent restarted (F)GMRES written here with
  plain numpy -- Arnoldi with classical Gram-Schmidt applied twice and the
  small least-squares problem solved by numpy's lstsq instead of Givens
  rotations -- must give the same residual after every inner step, the same
  iteration count and the same solution.
* The singular l-AIR local system (Section 3: each C point solves
  A_ff(N_i, N_i)^T z = -A(i, N_i)^T).  When that block is singular to working
  precision the oracle keeps injection, z = 0, and counts the system.  A hand
  built matrix whose local block is exactly singular checks the row and the
  count, and a nonsingular twin checks that the branch is not taken there.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from sthdg import assemble
from sthdg.problems import manufactured_2d


def _sp(rp, ci, v, n):
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


def _restarted_fgmres(A, b, m, rtol, max_iter, prec=None):
    """Restarted right-preconditioned flexible GMRES from x0 = 0, written from
    the textbook definition: each cycle minimises ||beta e1 - Hbar y|| over the
    Krylov space of the current residual.  The stopping rule is the oracle's:
    the true residual decides at the start of every cycle, the least-squares
    residual inside a cycle.  Returns (x, iters, per-step relative residuals,
    true relative residual at exit)."""
    n = len(b)
    bn = np.linalg.norm(b)
    x = np.zeros(n)
    hist = [1.0]
    it = 0
    while True:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta / bn <= rtol or it >= max_iter:
            return x, it, np.array(hist), beta / bn
        V = np.zeros((n, m + 1))
        Z = np.zeros((n, m))
        Hb = np.zeros((m + 1, m))
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            if it >= max_iter:
                break
            Z[:, j] = V[:, j] if prec is None else prec(V[:, j])
            w = A @ Z[:, j]
            for _ in range(2):                      # classical Gram-Schmidt, twice
                h = V[:, :j + 1].T @ w
                w = w - V[:, :j + 1] @ h
                Hb[:j + 1, j] += h
            Hb[j + 1, j] = np.linalg.norm(w)
            if Hb[j + 1, j] > 0:
                V[:, j + 1] = w / Hb[j + 1, j]
            k = j + 1
            it += 1
            e1 = np.zeros(k + 1)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(Hb[:k + 1, :k], e1, rcond=None)
            res = np.linalg.norm(e1 - Hb[:k + 1, :k] @ y) / bn
            hist.append(res)
            if res <= rtol or Hb[j + 1, j] == 0:
                break
        e1 = np.zeros(k + 1)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(Hb[:k + 1, :k], e1, rcond=None)
        x = x + Z[:, :k] @ y


@pytest.fixture(scope="module")
def sys_small():
    # 2D+time, n = 3, p = 1, nu = 1e-2: 1,296 unknowns, nonsymmetric
    return assemble(manufactured_2d(3, 1, 1e-2))


def _close_hist(h_oracle, h_ref):
    # the two residual sequences agree to rounding; once they fall to ~1e-12
    # of ||b|| their own rounding dominates, hence the absolute floor
    assert len(h_oracle) == len(h_ref)
    diff = np.abs(h_oracle - h_ref)
    assert np.all(diff <= 1e-7 * h_ref + 1e-11), np.max(diff / (h_ref + 1e-30))


@pytest.mark.parametrize("m", [2, 5])
def test_gmres_restart_unpreconditioned_matches_independent(sys_small, m):
    s = sys_small
    A = _sp(s.row_ptr, s.col, s.val, s.n)
    x, it, rr, ok, hist = oracle.gmres(s.row_ptr, s.col, s.val, None, s.rhs, rtol=1e-9, restart=m,
                                       max_iter=3000)
    xr, itr, histr, rrr = _restarted_fgmres(A, s.rhs, m, 1e-9, 3000)
    assert ok and it > 3 * m                  # several restart cycles were taken
    assert it == itr
    _close_hist(hist, histr)
    assert abs(rr - rrr) <= 1e-7 * rrr + 1e-13
    xd = np.linalg.solve(A.toarray(), s.rhs)
    assert np.linalg.norm(s.rhs - A @ x) <= 1e-9 * np.linalg.norm(s.rhs) * 1.0001
    assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xd)


@pytest.mark.parametrize("m", [3, 4])
def test_fgmres_restart_with_vcycle_matches_independent(m):
    """Preconditioned: Z_j = M^{-1} V_j with one oracle V-cycle as M^{-1}; after
    a restart the update must use Z (not V), which only a preconditioned run
    can tell apart."""
    s = assemble(manufactured_2d(4, 1, 1e-4))
    A = _sp(s.row_ptr, s.col, s.val, s.n)
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    x, it, rr, ok, hist = oracle.gmres(s.row_ptr, s.col, s.val, H, s.rhs, rtol=1e-10, restart=m, max_iter=500)
    xr, itr, histr, rrr = _restarted_fgmres(A, s.rhs, m, 1e-10, 500, prec=H.vcycle)
    assert ok and it > 2 * m
    assert it == itr
    _close_hist(hist, histr)
    xd = np.linalg.solve(A.toarray(), s.rhs)
    assert np.linalg.norm(s.rhs - A @ x) <= 1e-10 * np.linalg.norm(s.rhs) * 1.0001
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)


def test_gmres_restart_stops_at_max_iter_mid_cycle(sys_small):
    """max_iter inside a cycle: the partial cycle is still applied to x, as in
    the reference implementation above."""
    s = sys_small
    A = _sp(s.row_ptr, s.col, s.val, s.n)
    x, it, rr, ok, _ = oracle.gmres(s.row_ptr, s.col, s.val, None, s.rhs, rtol=1e-14, restart=5, max_iter=13)
    xr, itr, _, rrr = _restarted_fgmres(A, s.rhs, 5, 1e-14, 13)
    assert not ok and it == 13 == itr
    assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)
    assert abs(rr - rrr) <= 1e-9 * rrr


# ------------------------------------------------------------ singular l-AIR
def _triples(singular):
    """Independent 3-point blocks, one per entry of `singular`.  Block rows
    (i = 3k + 0, 1, 2):
        [ 3 -1 -1 ]      every off-diagonal is strong (theta = 0.25), every
        [-1  d  1 ]      measure |S^T_i| is 2, so the first point of each block
        [-1  c  1 ]      is picked C and the other two become F.
    The C point's local system is A_ff(N, N)^T with N = the two F points:
    [[d, c], [1, 1]]: exactly singular for d = c = 1, of determinant 3/2 for
    d = 2, c = 1/2 (then z = (1/3, 2/3)).  The first row's sum keeps the
    coarse operator nonsingular."""
    blocks = [np.array([[3.0, -1.0, -1.0], [-1.0, 1.0 if sg else 2.0, 1.0], [-1.0, 1.0 if sg else 0.5, 1.0]])
              for sg in singular]
    M = sp.csr_matrix(sp.block_diag(blocks, format="csr"))
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64)


def test_lair_singular_local_system_gives_injection_row():
    rp, ci, v = _triples([True])
    H = oracle.setup(rp, ci, v, theta=0.25, max_coarse=1, max_levels=2)
    L = H.levels[0]
    assert list(L.cf) == [1, 0, 0]
    assert L.n_singular == 1 and L.max_m == 2
    Rrp, Rci, Rv = L.R
    assert list(Rrp) == [0, 3] and list(Rci) == [0, 1, 2]
    assert list(Rv) == [1.0, 0.0, 0.0]               # injection: z = 0
    # injection with one-point P (weight 1): the coarse operator is row 0's sum
    assert H.levels[1].A[2].tolist() == [1.0]


def test_lair_nonsingular_twin_solves_the_local_system():
    rp, ci, v = _triples([False])
    H = oracle.setup(rp, ci, v, theta=0.25, max_coarse=1, max_levels=2)
    L = H.levels[0]
    assert list(L.cf) == [1, 0, 0] and L.n_singular == 0
    A = _sp(rp, ci, v, 3).toarray()
    # z solves A_ff^T z = -A(0, F)^T, i.e. (R A)(0, F) = 0
    z = np.linalg.solve(A[1:, 1:].T, -A[0, 1:])
    assert np.allclose(L.R[2], [1.0, *z], rtol=1e-15, atol=1e-15)
    RA = L.R[2] @ A
    assert np.allclose(RA[1:], 0.0, atol=1e-15)


def test_lair_singular_count_over_many_blocks():
    rp, ci, v = _triples([k % 2 == 0 for k in range(40)])
    H = oracle.setup(rp, ci, v, theta=0.25, max_coarse=1, max_levels=2)
    L = H.levels[0]
    assert L.n_singular == 20 and L.nc == 40
    Rv = L.R[2].reshape(40, 3)
    assert np.all(Rv[0::2, 1:] == 0.0)               # singular blocks: injection
    assert np.all(Rv[1::2, 1:] != 0.0)               # the others: the local solve


# ------------------------------------------------------------ distance-2 l-AIR
def test_lair_distance2_neighbourhoods_and_invariant():
    """Distance two (Section 3: l-AIR with larger neighbourhoods): N_i is the
    strongly connected F points of i and of those F points, recomputed here
    from the definition; R's columns are N_i plus i and (R A)(i, N_i) = 0."""
    s = assemble(manufactured_2d(3, 2, 1e-2))
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, distance=2, max_coarse=50, max_levels=3)
    for l, L in enumerate(H.levels[:-1]):
        Srp, Sci = L.S
        S = [set(Sci[Srp[i]:Srp[i + 1]].tolist()) for i in range(L.n)]
        F = set(np.nonzero(L.cf == 0)[0].tolist())
        A = _sp(*L.A, L.n)
        Rrp, Rci, Rv = L.R
        R = sp.csr_matrix((Rv, Rci, Rrp), shape=(L.nc, L.n))
        RA = (R @ A).tocsr()
        for r, i in enumerate(np.nonzero(L.cf == 1)[0]):
            N1 = S[i] & F
            N = set(N1)
            for k in N1:
                N |= S[k] & F
            cols = Rci[Rrp[r]:Rrp[r + 1]].tolist()
            assert cols == sorted(N | {int(i)})
            row = RA.getrow(r).toarray()[0]
            if N:
                scale = np.abs(A[sorted(N)][:, sorted(N)]).max()
                assert np.max(np.abs(row[sorted(N)])) <= 1e-12 * scale * max(1.0, np.abs(Rv[Rrp[r]:Rrp[r + 1]]).max())
    assert max(L.max_m for L in H.levels[:-1]) > max(
        oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, distance=1, max_coarse=50, max_levels=3).levels[0].max_m, 0)
