"""air_gmres_solve_noalloc against air_gmres_solve, through the C ABI.

The allocation-free solve serves callers that cannot let the library allocate
device memory during the solve (memory fully pre-assigned by a pool or a
budget, or a framework that forbids allocation inside its solve phase).  It
runs the same kernels on a fixed device array, so on the same hierarchy it
must reproduce the allocating solve -- here twice in a row, since the array
keeps the previous call's contents.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2010_11130_gb300 as air  # noqa: E402
from paper_2010_11130_gb300.air import gmres_solve_noalloc  # noqa: E402
from sthdg import assemble  # noqa: E402
from sthdg.problems import manufactured_1d, manufactured_2d  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    air.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_allocating_solve_twice(precision):
    s = assemble(manufactured_2d(6, 2, 1e-6))          # 15,120 unknowns
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, precision=precision)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x_ref, info_ref = air.gmres_solve(A, H, b, rtol=1e-8)
    torch.cuda.synchronize()
    for _ in range(2):
        x = torch.full_like(b, 7.0)                    # garbage: the solve must overwrite it
        x, info = gmres_solve_noalloc(A, H, b, x, rtol=1e-8)
        torch.cuda.synchronize()
        assert info.status == 0
        assert info.iters == info_ref.iters
        assert abs(info.relres - info_ref.relres) <= 1e-12
        xr = x_ref.cpu().numpy()
        assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-12 * np.linalg.norm(xr)


def test_noalloc_second_problem_after_first():
    # a different, smaller system after a larger one: stale workspace contents must not leak
    s = assemble(manufactured_1d(16, 1, 1e-4))
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x_ref, info_ref = air.gmres_solve(A, H, b, rtol=1e-8)
    x, info = gmres_solve_noalloc(A, H, b, torch.empty_like(b), rtol=1e-8)
    torch.cuda.synchronize()
    assert info.iters == info_ref.iters
    assert np.linalg.norm(x.cpu().numpy() - x_ref.cpu().numpy()) <= 1e-12 * np.linalg.norm(x_ref.cpu().numpy())


def test_noalloc_rejects_problems_beyond_the_workspace():
    s = assemble(manufactured_2d(10, 2, 1e-6))         # 70,800 unknowns > the fixed workspace
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=1000)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    with pytest.raises(air.AirError) as e:
        gmres_solve_noalloc(A, H, b, torch.empty_like(b), rtol=1e-8)
    assert e.value.status == -9
