"""Degenerate and ragged inputs through the C ABI, against the oracle.

The method's degenerate cases: a single unknown; a matrix with no
off-diagonal entries (no strong connections, so every point is F, nothing
coarsens and level 0 is the coarsest, solved by its dense inverse, or an error
when it exceeds max_dense); isolated rows inside a coupled system (points
with S_i and S^T_i empty start F); a zero right-hand side; a row with no
entries (rejected: the relaxation needs a_ii); and tiny chains whose sizes
cut SELL-32 slices, neighbourhood blocks and bitmap words raggedly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2010_11130_gb300 as air  # noqa: E402
from sthdg import assemble  # noqa: E402
from sthdg.problems import manufactured_2d  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    air.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _levels_match_oracle(H, O):
    assert H.levels() == len(O.levels)
    for l, OL in enumerate(O.levels):
        assert np.array_equal(H.export(l, "A.val"), OL.A[2])
        if OL.nc == 0:
            assert H.info(l).coarsest == 1
            continue
        assert np.array_equal(H.export(l, "cf"), OL.cf)
        assert np.array_equal(H.export(l, "R.col"), OL.R[1])
        assert np.array_equal(H.export(l, "R.val"), OL.R[2])
        assert np.array_equal(H.export(l, "pcol"), OL.pcol)


def _chain(n, seed):
    """Lower-bidiagonal upwind chain with random positive diagonal and negative
    subdiagonal (every row but the first has one strong connection)."""
    rng = np.random.default_rng(seed)
    rp = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        if i > 0:
            cols.append(i - 1)
            vals.append(-(0.5 + rng.random()))
        cols.append(i)
        vals.append(1.0 + rng.random())
        rp[i + 1] = len(cols)
    return rp, np.array(cols, dtype=np.int32), np.array(vals)


def test_single_unknown():
    rp, ci, v = np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), np.array([4.0])
    A = air.CSR.from_host(rp, ci, v)
    H = air.setup(A)
    assert H.levels() == 1 and H.info(0).coarsest == 1
    x = H.vcycle(_dev([2.0]))
    torch.cuda.synchronize()
    assert float(x[0]) == 0.5
    x, info = air.gmres_solve(A, H, _dev([2.0]), rtol=1e-12)
    assert info.status == 0 and info.iters <= 1 and abs(float(x[0]) - 0.5) <= 1e-15


@pytest.mark.parametrize("precision", [0, 1])
def test_diagonal_matrix_is_its_own_coarsest_level(precision):
    n = 1200
    rng = np.random.default_rng(3)
    d = 1.0 + rng.random(n)
    rp, ci = np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32)
    A = air.CSR.from_host(rp, ci, d)
    H = air.setup(A, max_coarse=100, precision=precision)
    O = oracle.setup(rp, ci, d, max_coarse=100)
    assert H.levels() == 1 == len(O.levels)
    b = rng.standard_normal(n)
    x = H.vcycle(_dev(b))
    torch.cuda.synchronize()
    tol = 1e-13 if precision == 0 else 1e-6
    assert np.linalg.norm(x.cpu().numpy() - b / d) <= tol * np.linalg.norm(b / d)
    assert np.linalg.norm(O.vcycle(b) - b / d) <= 1e-13 * np.linalg.norm(b / d)
    x, info = air.gmres_solve(A, H, _dev(b), rtol=1e-10)
    assert info.status == 0 and info.iters <= 2


def test_uncoarsenable_level_above_max_dense_is_an_error():
    n = 1200
    rp, ci = np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32)
    A = air.CSR.from_host(rp, ci, np.full(n, 2.0))
    with pytest.raises(air.AirError) as e:
        air.setup(A, max_coarse=100, max_dense=1000)
    assert e.value.status == -7
    with pytest.raises(oracle.OracleError):
        oracle.setup(rp, ci, np.full(n, 2.0), max_coarse=100, max_dense=1000)


def test_isolated_rows_inside_a_coupled_system():
    # a 2D+time trace system with 37 decoupled rows appended (ragged tail):
    # the isolated points start F and the rest coarsens as before
    s = assemble(manufactured_2d(5, 2, 1e-6))
    k = 37
    n = s.n + k
    rp = np.concatenate([s.row_ptr, s.row_ptr[-1] + np.arange(1, k + 1, dtype=np.int64)])
    ci = np.concatenate([s.col, np.arange(s.n, n, dtype=np.int32)])
    v = np.concatenate([s.val, 1.0 + np.arange(k) / k])
    A = air.CSR.from_host(rp, ci, v)
    H = air.setup(A, max_coarse=100)
    O = oracle.setup(rp, ci, v, max_coarse=100)
    _levels_match_oracle(H, O)
    cf = H.export(0, "cf")
    assert np.all(cf[s.n:] == 0)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(n)
    x = H.vcycle(_dev(b))
    torch.cuda.synchronize()
    xo = O.vcycle(b)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)
    x, info = air.gmres_solve(A, H, _dev(b), rtol=1e-8)
    _, it, _, conv, _ = oracle.gmres(rp, ci, v, O, b, rtol=1e-8)
    assert conv and abs(info.iters - it) <= 1


def test_zero_right_hand_side():
    s = assemble(manufactured_2d(4, 1, 1e-4))
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    for precision in (0, 1, 2):
        H = air.setup(A, max_coarse=50, precision=precision)
        x, info = air.gmres_solve(A, H, torch.zeros(s.n, dtype=torch.float64, device="cuda"), rtol=1e-8)
        torch.cuda.synchronize()
        assert info.status == 0 and info.iters == 0 and float(x.abs().max()) == 0.0


def test_row_without_entries_is_rejected():
    rp = np.array([0, 2, 2, 3], dtype=np.int64)           # row 1 is empty
    ci = np.array([0, 2, 2], dtype=np.int32)
    with pytest.raises(air.AirError) as e:
        air.setup(air.CSR.from_host(rp, ci, np.array([1.0, 0.5, 1.0])))
    assert e.value.status == -2


@pytest.mark.parametrize("n", [2, 31, 33, 63, 65, 511, 513, 4097])
def test_ragged_chains_match_oracle(n):
    rp, ci, v = _chain(n, seed=n)
    A = air.CSR.from_host(rp, ci, v)
    H = air.setup(A, max_coarse=2)
    O = oracle.setup(rp, ci, v, max_coarse=2)
    _levels_match_oracle(H, O)
    b = np.random.default_rng(n + 1).standard_normal(n)
    x = H.vcycle(_dev(b))
    torch.cuda.synchronize()
    xo = O.vcycle(b)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)
