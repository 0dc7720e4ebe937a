"""GPU GMRES across restart cycles and the singular l-AIR branch, against the
oracle, through the C ABI.

The benchmark's solve takes about four GMRES(30) cycles, so the restart path
(H y = g, x += Z y, a new Arnoldi cycle from the true residual b - A x) is
compared here: with a short restart length on the parity systems, and at the
default length on a system that needs more than 30 iterations.  Iteration
counts within one of the oracle's, the true residual at the tolerance
(re-checked with the oracle's SpMV) and the solution near the oracle's.

The l-AIR local systems (Section 3) of a hand-built matrix are exactly
singular for half of its C points: the GPU must take the oracle's injection
row (z = 0) there, count the systems alike and agree bit for bit elsewhere.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2010_11130_gb300 as air  # noqa: E402
from paper_2010_11130_gb300.air import gmres_solve_noalloc  # noqa: E402
from sthdg import assemble  # noqa: E402
from sthdg.problems import manufactured_1d, manufactured_2d  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    air.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


_CASES = {
    "st1d_n32_p1": lambda: assemble(manufactured_1d(32, 1, 1e-4)),
    "st2d_n6_p2_nu1e-6": lambda: assemble(manufactured_2d(6, 2, 1e-6)),
    "st2d_n8_p1_nu1e-2": lambda: assemble(manufactured_2d(8, 1, 1e-2)),
    "st2d_n5_p3_nu1e-5": lambda: assemble(manufactured_2d(5, 3, 1e-5)),
}
_cache = {}


def _system(name):
    if name not in _cache:
        _cache[name] = _CASES[name]()
    return _cache[name]


def _check_solution(s, x, info, xo, ito, rtol):
    assert info.status == 0
    assert abs(info.iters - ito) <= 1, (info.iters, ito)
    r = s.rhs - oracle.spmv(s.row_ptr, s.col, s.val, x)
    assert np.linalg.norm(r) <= rtol * np.linalg.norm(s.rhs) * (1 + 1e-6)
    assert abs(info.relres - np.linalg.norm(r) / np.linalg.norm(s.rhs)) <= 1e-12
    # both residuals are below rtol; the solutions differ by at most about
    # cond(A) rtol, and these systems are well conditioned after block scaling
    assert np.linalg.norm(x - xo) <= 1e3 * rtol * np.linalg.norm(xo)


@pytest.mark.parametrize("restart", [4, 5])
@pytest.mark.parametrize("name", list(_CASES.keys()))
def test_gmres_short_restart_matches_oracle(name, restart):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, restart=restart)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.gmres_solve(A, H, b, rtol=1e-8)
    torch.cuda.synchronize()
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    xo, ito, rro, oko, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-8, restart=restart)
    assert oko and ito > 2 * restart                 # at least two restarts taken
    assert info.restarts >= 3
    _check_solution(s, x.cpu().numpy(), info, xo, ito, 1e-8)


@pytest.mark.parametrize("precision", [1, 2])
def test_fgmres_low_precision_hierarchy_across_restarts(precision):
    """FP32 / BF16-off-diagonal hierarchies inside FP64 flexible GMRES(5): the
    outer loop still reaches 1e-10 across several cycles."""
    s = _system("st2d_n6_p2_nu1e-6")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, restart=5, precision=precision)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.gmres_solve(A, H, b, rtol=1e-10)
    torch.cuda.synchronize()
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    xo, ito, _, _, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-10, restart=5)
    assert info.status == 0 and info.relres <= 1e-10 and info.restarts >= 3
    assert info.iters <= ito + (3 if precision == 1 else 10)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-7 * np.linalg.norm(xo)


def test_gmres30_beyond_one_cycle_on_571k_unknowns():
    """2D+time n = 20, p = 2, nu = 1e-6 (571,200 unknowns): the oracle needs
    more than 30 iterations, so GMRES(30) restarts at least once."""
    s = assemble(manufactured_2d(20, 2, 1e-6), workers=8)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=1000)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.gmres_solve(A, H, b, rtol=1e-8)
    torch.cuda.synchronize()
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=1000)
    xo, ito, _, oko, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-8)
    assert oko and ito > 30
    assert info.restarts >= 1
    _check_solution(s, x.cpu().numpy(), info, xo, ito, 1e-8)


def test_noalloc_across_restarts_matches_allocating_solve():
    s = _system("st2d_n6_p2_nu1e-6")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, restart=5)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x_ref, info_ref = air.gmres_solve(A, H, b, rtol=1e-8)
    x, info = gmres_solve_noalloc(A, H, b, torch.full_like(b, 3.0), rtol=1e-8)
    torch.cuda.synchronize()
    assert info_ref.restarts >= 3
    assert info.iters == info_ref.iters and info.restarts == info_ref.restarts
    xr = x_ref.cpu().numpy()
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-12 * np.linalg.norm(xr)


# ------------------------------------------------------------ singular l-AIR
def _triples(singular):
    """Independent 3-point blocks [[3,-1,-1],[-1,d,1],[-1,c,1]]: the first point
    of each is C, the other two F, and the C point's local system
    [[d, c], [1, 1]] is exactly singular for d = c = 1 (and has z = (1/3, 2/3)
    for d = 2, c = 1/2)."""
    blocks = [np.array([[3.0, -1.0, -1.0], [-1.0, 1.0 if sg else 2.0, 1.0], [-1.0, 1.0 if sg else 0.5, 1.0]])
              for sg in singular]
    M = sp.csr_matrix(sp.block_diag(blocks, format="csr"))
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64)


def test_singular_local_systems_bit_exact():
    rp, ci, v = _triples([k % 2 == 0 for k in range(1000)])
    A = air.CSR.from_host(rp, ci, v)
    H = air.setup(A, theta=0.25, max_coarse=100)
    O = oracle.setup(rp, ci, v, theta=0.25, max_coarse=100)
    assert H.levels() == len(O.levels)
    OL = O.levels[0]
    assert OL.n_singular == 500
    assert H.info(0).n_singular == 500
    assert np.array_equal(H.export(0, "cf"), OL.cf)
    assert np.array_equal(H.export(0, "R.col"), OL.R[1])
    assert np.array_equal(H.export(0, "R.val"), OL.R[2])
    assert np.array_equal(H.export(1, "A.val"), O.levels[1].A[2])
    b = np.random.default_rng(7).standard_normal(len(rp) - 1)
    x = H.vcycle(torch.from_numpy(b).cuda())
    torch.cuda.synchronize()
    xo = O.vcycle(b)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)
