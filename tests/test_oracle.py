"""Pins of the CPU oracle (oracle/air_oracle.c) against what the paper and the
mathematics fix: closed forms, invariants, brute force on tiny inputs and
dense-matrix definitions (Section 3: two-level correction, ideal restriction;
Section 4 settings: strength, one-point interpolation, relaxation)."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from sthdg import assemble
from sthdg.problems import manufactured_1d, manufactured_2d, pure_advection


def _sp(rp, ci, v, shape):
    return sp.csr_matrix((v, ci, rp), shape=shape)


def _dense_csr(M):
    S = sp.csr_matrix(M)
    S.sort_indices()
    return S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64)


@pytest.fixture(scope="module")
def sys1d():
    return assemble(manufactured_1d(8, 1, 1e-3))


@pytest.fixture(scope="module")
def sys2d():
    return assemble(manufactured_2d(4, 1, 1e-4))


def test_spmv_matches_scipy(sys2d):
    s = sys2d
    x = np.random.default_rng(0).standard_normal(s.n)
    y = oracle.spmv(s.row_ptr, s.col, s.val, x)
    assert np.allclose(y, _sp(s.row_ptr, s.col, s.val, (s.n, s.n)) @ x, rtol=1e-14, atol=1e-14)


def test_strength_hand_built():
    # row 0: off-diag |.| = 4, 1, 2 -> theta=0.25: threshold 1 -> {1, 2, 3}
    # row 1: off-diag 0.5, 0.1       -> threshold 0.125 -> {0}
    # row 2: no off-diagonal          -> {}
    # row 3: off-diag -3, 3           -> ties kept: {0, 2}
    M = np.array([[1.0, -4.0, 1.0, 2.0],
                  [0.5, 1.0, 0.0, 0.1],
                  [0.0, 0.0, 1.0, 0.0],
                  [-3.0, 0.0, 3.0, 1.0]])
    # a dense 4x4 has to stay above max_coarse to be coarsened: use max_coarse=0
    H = oracle.setup(*_dense_csr(M), theta=0.25, max_coarse=0, max_levels=2)
    rp, ci = H.levels[0].S
    rows = [list(ci[rp[i]:rp[i + 1]]) for i in range(4)]
    assert rows == [[1, 2, 3], [0], [], [0, 2]]


def _chain(n):
    """1D first-order upwind chain: x_i - x_{i-1} = b_i."""
    return sp.diags([np.ones(n), -np.ones(n - 1)], [0, -1]).toarray()


@pytest.mark.parametrize("n", [10, 11])
def test_rs_on_upwind_chain(n):
    """Closed form of the first pass on a chain: C at even, F at odd indices;
    an even last point has measure 0 and ends F."""
    H = oracle.setup(*_dense_csr(_chain(n)), theta=0.25, max_coarse=0, max_levels=2)
    cf = H.levels[0].cf
    want = np.array([1 if i % 2 == 0 else 0 for i in range(n)], dtype=np.int8)
    if n % 2 == 1:
        want[-1] = 0
    assert np.array_equal(cf, want)


def _rs_bruteforce(S):
    """First-pass C/F splitting written from its definition with O(n^2) scans."""
    n = len(S)
    ST = [[i for i in range(n) if j in S[i]] for j in range(n)]
    lam = [len(ST[i]) for i in range(n)]
    state = ["U"] * n
    for i in range(n):
        if not S[i] and not ST[i]:
            state[i] = "F"
    while True:
        cand = [i for i in range(n) if state[i] == "U"]
        if not cand:
            break
        best = max(cand, key=lambda i: (lam[i], -i))
        if lam[best] == 0:
            break
        state[best] = "C"
        for j in ST[best]:
            if state[j] == "U":
                state[j] = "F"
                for k in S[j]:
                    if state[k] == "U":
                        lam[k] += 1
        for k in S[best]:
            if state[k] == "U":
                lam[k] -= 1
    return np.array([1 if s == "C" else 0 for s in state], dtype=np.int8)


@pytest.mark.parametrize("seed", range(40))
def test_rs_matches_bruteforce_small_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 13))
    M = np.eye(n) * 4.0
    mask = rng.random((n, n)) < 0.3
    np.fill_diagonal(mask, False)
    M[mask] = -rng.choice([1.0, 1.0, 2.0], size=mask.sum())   # ties in |a| on purpose
    H = oracle.setup(*_dense_csr(M), theta=0.25, max_coarse=0, max_levels=2)
    rp, ci = H.levels[0].S if H.levels[0].S is not None else (None, None)
    if rp is None:       # no coarsening happened: every point F or nothing strong
        return
    S = [list(ci[rp[i]:rp[i + 1]]) for i in range(n)]
    assert np.array_equal(H.levels[0].cf, _rs_bruteforce(S))


def _level_mats(L, n_next):
    n = L.n
    A = _sp(*L.A, (n, n))
    R = _sp(*L.R, (L.nc, n))
    rows = np.nonzero(L.pcol >= 0)[0]
    P = sp.csr_matrix((L.pw[rows], (rows, L.pcol[rows])), shape=(n, n_next))
    return A, R, P


def test_lair_invariant_RA_zero_on_neighbourhood(sys2d):
    """(R A)(i, j) = 0 for j in N_i: the defining local condition of l-AIR."""
    s = sys2d
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=50)
    for l, L in enumerate(H.levels[:-1]):
        A, R, P = _level_mats(L, H.levels[l + 1].n)
        RA = (R @ A).tocsr()
        Cpts = np.nonzero(L.cf == 1)[0]
        worst = 0.0
        for r, i in enumerate(Cpts):
            Ni = [j for j in R.indices[R.indptr[r]:R.indptr[r + 1]] if j != i]
            if not Ni:
                continue
            vals = RA[r, Ni].toarray().ravel()
            scale = np.abs(A[i]).max()
            worst = max(worst, np.abs(vals).max() / scale)
        assert worst < 1e-12


def test_onepoint_P_definition(sys2d):
    s = sys2d
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=50)
    L = H.levels[0]
    A = _sp(*L.A, (L.n, L.n))
    Srp, Sci = L.S
    for i in range(L.n):
        if L.cf[i] == 1:
            assert L.pcol[i] == L.cid[i] and L.pw[i] == 1.0
            continue
        strongC = [j for j in Sci[Srp[i]:Srp[i + 1]] if L.cf[j] == 1]
        if not strongC:
            assert L.pcol[i] == -1
            continue
        mags = np.abs(A[i, strongC].toarray().ravel())
        best = strongC[int(np.flatnonzero(mags == mags.max())[0])]
        assert L.pcol[i] == L.cid[best] and L.pw[i] == 1.0


def test_first_pass_f_points_invariant(sys2d):
    """Measure bookkeeping of the first pass: lambda_j counts undecided strong
    dependants once, F dependants twice and C dependants not at all, so an F
    point that ends without a strong C neighbour (it was never made F by a C
    pick) must have had only C points among its strong dependants S^T_j."""
    s = sys2d
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=50)
    L = H.levels[0]
    Srp, Sci = L.S
    ST = sp.csr_matrix((np.ones(len(Sci)), Sci, Srp), shape=(L.n, L.n)).T.tocsr()
    lonely = 0
    for j in np.nonzero(L.cf == 0)[0]:
        if np.any(L.cf[Sci[Srp[j]:Srp[j + 1]]] == 1):
            continue
        lonely += 1
        deps = ST.indices[ST.indptr[j]:ST.indptr[j + 1]]
        assert np.all(L.cf[deps] == 1)
    assert np.sum(L.cf == 1) > 0


def test_rap_equals_dense_triple_product(sys1d):
    s = sys1d
    assert s.n <= 600
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=20)
    assert len(H.levels) >= 3
    for l, L in enumerate(H.levels[:-1]):
        A, R, P = _level_mats(L, H.levels[l + 1].n)
        dense = R.toarray() @ A.toarray() @ P.toarray()
        nxt = H.levels[l + 1]
        Ac = _sp(*nxt.A, (nxt.n, nxt.n)).toarray()
        assert np.allclose(Ac, dense, rtol=1e-13, atol=1e-13 * np.abs(dense).max())
        # structural pattern contains every nonzero of the product
        assert np.all((np.abs(dense) > 1e-12 * np.abs(dense).max()) <= (_sp(*nxt.A, (nxt.n, nxt.n)).toarray() != 0)
                      | (np.abs(dense) <= 1e-12 * np.abs(dense).max()))


def _dense_vcycle_operator(H, relax="FCF", omega=1.0):
    """M^{-1} as a dense matrix, composed from the level operators by the
    definition of the V-cycle (zero initial guess, restriction, exact coarsest
    solve, interpolation, Jacobi sweeps)."""
    def level_op(l):
        L = H.levels[l]
        A = _sp(*L.A, (L.n, L.n)).toarray()
        if l == len(H.levels) - 1:
            return np.linalg.inv(A)
        _, R, P = _level_mats(L, H.levels[l + 1].n)
        R, P = R.toarray(), P.toarray()
        M = P @ level_op(l + 1) @ R           # x = P A_c^{-1} R b
        d = np.diag(A)
        I = np.eye(L.n)
        for c in relax:
            mask = (L.cf == (1 if c == "C" else 0)).astype(float)
            Dm = np.diag(mask * omega / d)
            # x <- x + D_S (b - A x)  =>  M <- M + D_S (I - A M)
            M = M + Dm @ (I - A @ M)
        return M
    return level_op(0)


def test_vcycle_equals_dense_composition(sys1d):
    s = sys1d
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=20)
    Minv = _dense_vcycle_operator(H)
    rng = np.random.default_rng(1)
    for _ in range(3):
        b = rng.standard_normal(s.n)
        assert np.allclose(H.vcycle(b), Minv @ b, rtol=1e-12, atol=1e-12 * np.abs(Minv @ b).max())


@pytest.mark.parametrize("D,n,p", [(2, 6, 1), (3, 2, 1)])
def test_exact_reduction_pure_advection(D, n, p):
    """nu = 0, triangular A_ff, every connection strong, distance covering the
    whole F-graph and F-relaxation iterated to exactness: R = R_ideal, the
    coarse-grid correction removes all C-point error and one V-cycle solves
    the system (ideal restriction property, Section 3)."""
    s = assemble(pure_advection(D, n, p))
    depth = s.n
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=1e-12, distance=s.n, max_coarse=0,
                     max_levels=2, max_dense=s.n, relax="F" * 40)
    L = H.levels[0]
    A = _sp(*L.A, (s.n, s.n)).toarray()
    # R equals R_ideal = [-A_cf A_ff^{-1}, I]
    F, Cp = np.nonzero(L.cf == 0)[0], np.nonzero(L.cf == 1)[0]
    Rid = np.zeros((len(Cp), s.n))
    Rid[:, F] = -A[np.ix_(Cp, F)] @ np.linalg.inv(A[np.ix_(F, F)])
    Rid[np.arange(len(Cp)), Cp] = 1.0
    R = _sp(*L.R, (L.nc, s.n)).toarray()
    assert np.allclose(R, Rid, atol=1e-12)
    x = H.vcycle(s.rhs)
    r = s.rhs - A @ x
    assert depth > 0
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(s.rhs)


def test_gmres_matches_dense_solve(sys2d):
    s = sys2d
    A = _sp(s.row_ptr, s.col, s.val, (s.n, s.n)).toarray()
    xd = np.linalg.solve(A, s.rhs)
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    x, it, rr, ok, hist = oracle.gmres(s.row_ptr, s.col, s.val, H, s.rhs, rtol=1e-10)
    assert ok and rr <= 1e-10
    assert np.linalg.norm(s.rhs - A @ x) <= 1e-10 * np.linalg.norm(s.rhs) * 1.0001
    cond = np.linalg.cond(A)
    assert np.linalg.norm(x - xd) <= cond * 1e-10 * np.linalg.norm(xd)
    assert np.all(np.diff(hist) <= 1e-15)          # GMRES residual is monotone


def test_gmres_unpreconditioned_small_exact():
    # GMRES on an n x n system converges in at most n steps (no restart)
    rng = np.random.default_rng(3)
    n = 12
    M = np.eye(n) * 3 + rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    x, it, rr, ok, _ = oracle.gmres(*_dense_csr(M), None, b, rtol=1e-12, restart=n, max_iter=n)
    assert ok and it <= n
    assert np.allclose(x, np.linalg.solve(M, b), rtol=1e-9)


def test_coarsening_stops_and_levels_shrink():
    s = assemble(manufactured_2d(6, 1, 1e-6))
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=200)
    ns = [L.n for L in H.levels]
    assert ns[-1] <= 200
    assert all(b < 0.9 * a for a, b in zip(ns[:-1], ns[1:]))


# ------------------------------------------------------------------ BiCGSTAB
def test_bicgstab_unpreconditioned_matches_dense_solve():
    """Without a preconditioner BiCGSTAB is the plain van der Vorst iteration:
    on a small nonsymmetric trace system it reaches the dense solution."""
    s = assemble(manufactured_2d(2, 1, 1e-2))
    x, it, rr, ok = oracle.bicgstab(s.row_ptr, s.col, s.val, None, s.rhs, rtol=1e-12, max_iter=2000)
    A = _sp(s.row_ptr, s.col, s.val, (s.n, s.n)).toarray()
    xd = np.linalg.solve(A, s.rhs)
    assert ok and rr <= 1e-12 and it > 1
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_bicgstab_with_exact_preconditioner_takes_one_iteration():
    """With M^{-1} = A^{-1} (the exact two-level reduction of pure advection,
    as in the test above) the first iteration gives p^ = A^{-1} b, alpha = 1,
    s = 0: BiCGSTAB stops after one iteration."""
    s = assemble(pure_advection(3, 2, 1))
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=1e-12, distance=s.n, max_coarse=0,
                     max_levels=2, max_dense=s.n, relax="F" * 40)
    x, it, rr, ok = oracle.bicgstab(s.row_ptr, s.col, s.val, H, s.rhs, rtol=1e-10)
    assert ok and it == 1 and rr <= 1e-10


def test_bicgstab_with_air_matches_scipy_solution(sys2d):
    """AIR-preconditioned BiCGSTAB solves the system to 1e-12 (Section 5.1 uses
    this tolerance); the solution agrees with scipy's unpreconditioned BiCGSTAB
    run to the same tolerance."""
    import scipy.sparse.linalg as spl
    s = sys2d
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    x, it, rr, ok = oracle.bicgstab(s.row_ptr, s.col, s.val, H, s.rhs, rtol=1e-12)
    assert ok and rr <= 1e-12
    A = _sp(s.row_ptr, s.col, s.val, (s.n, s.n))
    xs, info = spl.bicgstab(A, s.rhs, rtol=1e-13, maxiter=20000)
    assert info == 0
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)


# ---------------------------------------------------- the paper's threshold pair
def test_theta_pair_equal_thresholds_is_the_single_threshold_setup(sys2d):
    s = sys2d
    H1 = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    H2 = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, theta_r=0.25, max_coarse=100)
    assert len(H1.levels) == len(H2.levels)
    for L1, L2 in zip(H1.levels, H2.levels):
        assert np.array_equal(L1.A[2], L2.A[2])
        if L1.R is not None:
            assert np.array_equal(L1.R[1], L2.R[1]) and np.array_equal(L1.R[2], L2.R[2])


def test_theta_pair_r_uses_its_own_strength_graph(sys2d):
    """Section 4: coarsening at strength 0.2, R from distance-one
    neighbourhoods at strength 0.3.  The splitting and P are those of the 0.2
    setup; every R row is {i} plus the F points strong for i at 0.3 (the
    classical definition, recomputed here from the matrix)."""
    s = sys2d
    Hc = oracle.setup(s.row_ptr, s.col, s.val, theta=0.2, max_coarse=100)
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.2, theta_r=0.3, max_coarse=100)
    L, Lc = H.levels[0], Hc.levels[0]
    assert np.array_equal(L.cf, Lc.cf) and np.array_equal(L.pcol, Lc.pcol)
    rp, ci, v = L.A
    Rp, Rc = L.R[0], L.R[1]
    C = np.nonzero(L.cf == 1)[0]
    differs = 0
    for r, i in enumerate(C):
        cols, vals = ci[rp[i]:rp[i + 1]], np.abs(v[rp[i]:rp[i + 1]])
        off = cols != i
        mx = vals[off].max() if off.any() else 0.0
        strong = cols[off & (vals >= 0.3 * mx)] if mx > 0 else np.array([], dtype=cols.dtype)
        want = np.sort(np.concatenate([[i], strong[L.cf[strong] == 0]]))
        got = Rc[Rp[r]:Rp[r + 1]]
        assert np.array_equal(got, want)
        differs += len(got) != Lc.R[0][r + 1] - Lc.R[0][r]
    assert differs > 0                      # the thresholds really select different neighbourhoods


def test_block_scaling_ablation():
    """Section 5.4: without the facet block-diagonal scaling ("No Block Inv") AIR
    loses its scalability.  With pointwise FCF-Jacobi relaxation the loss is
    total: the unscaled system is not solved in 200 iterations, the scaled
    one in under 30 (same mesh, same settings)."""
    res = {}
    for scale in (True, False):
        s = assemble(manufactured_2d(4, 2, 1e-6), scale=scale)
        H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
        _, it, _, ok, _ = oracle.gmres(s.row_ptr, s.col, s.val, H, s.rhs, rtol=1e-8, max_iter=200)
        _, itb, _, okb = oracle.bicgstab(s.row_ptr, s.col, s.val, H, s.rhs, rtol=1e-8, max_iter=200)
        res[scale] = (it, ok, itb, okb)
    assert res[True][1] and res[True][0] < 30 and res[True][3] and res[True][2] < 30
    assert not res[False][1] and not res[False][3]
