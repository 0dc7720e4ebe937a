"""Adjoint path on the GPU through the C ABI, against the oracle and dense solves.

air_csr_transpose / air_csr_outer and the differentiable solve of
paper_2010_11130_gb300.AdjointSolver: A^T is moved bit for bit, the l-AIR
hierarchy of A^T matches the oracle's bit for bit, and the autograd gradients
match the dense-LU gradient and central finite differences.
"""
import numpy as np
import pytest
import scipy.sparse as sp

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


_cache = {}


def _sys(n, p, nu):
    key = (n, p, nu)
    if key not in _cache:
        _cache[key] = assemble(manufactured_2d(n, p, nu))
    return _cache[key]


def _scipy(s):
    return sp.csr_matrix((s.val, s.col, s.row_ptr), shape=(s.n, s.n))


def test_transpose_bit_exact_against_scipy():
    s = _sys(6, 2, 1e-6)
    At = _scipy(s).T.tocsr()
    At.sort_indices()
    T = air.transpose(air.CSR.from_host(s.row_ptr, s.col, s.val))
    torch.cuda.synchronize()
    assert np.array_equal(T.row_ptr.cpu().numpy(), At.indptr)
    assert np.array_equal(T.col.cpu().numpy(), At.indices)
    assert np.array_equal(T.val.cpu().numpy(), At.data)


def test_transpose_of_unstructured_pattern():
    # a random non-symmetric pattern with empty rows and columns
    rng = np.random.default_rng(7)
    M = sp.random(700, 700, density=0.01, random_state=8, format="csr")
    M.setdiag(1.0 + rng.random(700))
    M = M.tocsr()
    M.sort_indices()
    T = air.transpose(air.CSR.from_host(M.indptr, M.indices, M.data))
    Mt = M.T.tocsr()
    Mt.sort_indices()
    assert np.array_equal(T.row_ptr.cpu().numpy(), Mt.indptr)
    assert np.array_equal(T.col.cpu().numpy(), Mt.indices)
    assert np.array_equal(T.val.cpu().numpy(), Mt.data)


def test_transpose_rejects_out_of_range_column():
    rp = np.array([0, 1, 2], dtype=np.int64)
    ci = np.array([0, 5], dtype=np.int32)          # column 5 of a 2 x 2 matrix
    A = air.CSR.from_host(rp, ci, np.ones(2))
    with pytest.raises(air.AirError) as e:
        air.transpose(A)
    assert e.value.status == -2


def test_csr_outer_matches_numpy():
    s = _sys(4, 2, 1e-6)
    rng = np.random.default_rng(2)
    u, w = rng.standard_normal(s.n), rng.standard_normal(s.n)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    out = air.csr_outer(A, torch.from_numpy(u).cuda(), torch.from_numpy(w).cuda(), -0.5)
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    ref = -0.5 * u[rows] * w[s.col]
    assert np.array_equal(out.cpu().numpy(), ref)


def test_adjoint_hierarchy_bit_exact_against_oracle():
    s = _sys(6, 2, 1e-6)
    At = _scipy(s).T.tocsr()
    At.sort_indices()
    rp, ci, v = At.indptr.astype(np.int64), At.indices.astype(np.int32), At.data.copy()
    T = air.transpose(air.CSR.from_host(s.row_ptr, s.col, s.val))
    H = air.setup(T, theta=0.25, max_coarse=100)
    O = oracle.setup(rp, ci, v, theta=0.25, max_coarse=100)
    assert H.levels() == len(O.levels)
    for l, OL in enumerate(O.levels):
        assert np.array_equal(H.export(l, "A.val"), OL.A[2])
        if OL.nc == 0:
            continue
        assert np.array_equal(H.export(l, "cf"), OL.cf)
        assert np.array_equal(H.export(l, "R.col"), OL.R[1])
        assert np.array_equal(H.export(l, "R.val"), OL.R[2])
    g = np.random.default_rng(4).standard_normal(s.n)
    lam, info = air.gmres_solve(T, H, torch.from_numpy(g).cuda(), rtol=1e-8)
    _, ito, _, oko, _ = oracle.gmres(rp, ci, v, O, g, rtol=1e-8)
    assert info.status == 0 and oko and abs(info.iters - ito) <= 1


def test_autograd_gradients_match_dense_lu():
    s = _sys(3, 2, 1e-2)
    rng = np.random.default_rng(9)
    ut = rng.standard_normal(s.n)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    A.val.requires_grad_(True)
    solver = air.AdjointSolver(A, rtol=1e-12)
    b = torch.from_numpy(s.rhs.copy()).cuda().requires_grad_(True)
    u = solver.solve(b)
    loss = 0.5 * torch.sum((u - torch.from_numpy(ut).cuda()) ** 2)
    loss.backward()
    D = _scipy(s).toarray()
    ud = np.linalg.solve(D, s.rhs)
    lam = np.linalg.solve(D.T, ud - ut)
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    gval = -lam[rows] * ud[s.col]
    gb = b.grad.cpu().numpy()
    gv = A.val.grad.cpu().numpy()
    assert np.linalg.norm(gb - lam) <= 1e-9 * np.linalg.norm(lam)
    assert np.linalg.norm(gv - gval) <= 1e-9 * np.linalg.norm(gval)
    assert solver.info.status == 0 and solver.info_adjoint.status == 0


def test_autograd_gradient_matches_central_differences():
    s = _sys(3, 2, 1e-6)
    rng = np.random.default_rng(13)
    ut = torch.from_numpy(rng.standard_normal(s.n)).cuda()
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    solver = air.AdjointSolver(A, rtol=1e-12)
    b0 = torch.from_numpy(s.rhs.copy()).cuda()

    def loss(b):
        return 0.5 * float(torch.sum((solver.solve(b) - ut) ** 2))

    b = b0.clone().requires_grad_(True)
    (0.5 * torch.sum((solver.solve(b) - ut) ** 2)).backward()
    g = b.grad.cpu().numpy()
    h = 1e-4      # L is quadratic in b: central differences are exact up to rounding
    for k in rng.choice(s.n, 3, replace=False):
        e = torch.zeros_like(b0)
        e[k] = h
        fd = (loss(b0 + e) - loss(b0 - e)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k]))


def test_adjoint_on_mapped_noisy_domain_matches_dense_lu():
    """The time-dependent mapped domain with noisy element velocities (its
    4^3 copy, dense LU as reference)."""
    from sthdg.problems import mapped_noisy
    s = assemble(mapped_noisy(4, 2, 1e-4))
    rng = np.random.default_rng(17)
    ut = rng.standard_normal(s.n)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    solver = air.AdjointSolver(A, rtol=1e-12)
    b = torch.from_numpy(s.rhs.copy()).cuda().requires_grad_(True)
    (0.5 * torch.sum((solver.solve(b) - torch.from_numpy(ut).cuda()) ** 2)).backward()
    D = _scipy(s).toarray()
    lam = np.linalg.solve(D.T, np.linalg.solve(D, s.rhs) - ut)
    assert np.linalg.norm(b.grad.cpu().numpy() - lam) <= 1e-9 * np.linalg.norm(lam)


def test_adjoint_on_mapped_noisy_8cubed_central_differences():
    from sthdg.problems import mapped_noisy
    s = assemble(mapped_noisy(8, 2, 1e-4))
    rng = np.random.default_rng(19)
    ut = torch.from_numpy(rng.standard_normal(s.n)).cuda()
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    solver = air.AdjointSolver(A, rtol=1e-12)
    b0 = torch.from_numpy(s.rhs.copy()).cuda()
    b = b0.clone().requires_grad_(True)
    (0.5 * torch.sum((solver.solve(b) - ut) ** 2)).backward()
    g = b.grad.cpu().numpy()
    h = 1e-4      # L is quadratic in b: central differences are exact up to rounding
    for k in rng.choice(s.n, 3, replace=False):
        e = torch.zeros_like(b0)
        e[k] = h
        lp = 0.5 * float(torch.sum((solver.solve(b0 + e) - ut) ** 2))
        lm = 0.5 * float(torch.sum((solver.solve(b0 - e) - ut) ** 2))
        assert abs((lp - lm) / (2 * h) - g[k]) <= 1e-6 * max(1.0, abs(g[k]))
