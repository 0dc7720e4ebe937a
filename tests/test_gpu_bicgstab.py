"""AIR-preconditioned BiCGSTAB on the GPU (air_bicgstab_solve) against the oracle.

The paper's experiments use BiCGSTAB to a relative residual of 1e-12
(Section 5.1, Table 2).  Parity bar: both converge, iteration counts within
one (dot products are reduced in a different order), true residual at the
tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2010_11130_gb300 as air  # noqa: E402
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


@pytest.mark.parametrize("name", list(_CASES))
def test_bicgstab_iterations_and_residual_match_oracle(name):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.bicgstab_solve(A, H, b, rtol=1e-12)
    torch.cuda.synchronize()
    xo, ito, rro, oko = oracle.bicgstab(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-12)
    assert info.status == 0 and oko
    assert abs(info.iters - ito) <= 1, (info.iters, ito)
    assert info.vcycles == 2 * info.iters
    r = s.rhs - oracle.spmv(s.row_ptr, s.col, s.val, x.cpu().numpy())
    rel = np.linalg.norm(r) / np.linalg.norm(s.rhs)
    assert rel <= 1e-12 * (1 + 1e-6)
    assert abs(info.relres - rel) <= 1e-14
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)


@pytest.mark.parametrize("precision", [1, 2])
def test_bicgstab_low_precision_hierarchy_converges(precision):
    # a fixed FP32 / BF16 V-cycle is a fixed linear preconditioner: BiCGSTAB
    # still reaches the FP64 tolerance, with a few more iterations
    s = _system("st2d_n6_p2_nu1e-6")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, precision=precision)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.bicgstab_solve(A, H, b, rtol=1e-10)
    assert info.status == 0 and info.relres <= 1e-10


def test_bicgstab_host_buffers_equal_device():
    s = _system("st1d_n32_p1")
    Ah = air.CSR(s.row_ptr.astype(np.int64), s.col.astype(np.int32), s.val.astype(np.float64), s.n)
    Hh = air.setup(Ah, theta=0.25, max_coarse=100)
    xh, ih = air.bicgstab_solve(Ah, Hh, np.ascontiguousarray(s.rhs), rtol=1e-12)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100)
    xd, idv = air.bicgstab_solve(A, H, torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda(), rtol=1e-12)
    assert ih.iters == idv.iters
    assert np.array_equal(xh, xd.cpu().numpy())


def test_bicgstab_zero_rhs_and_iteration_cap():
    s = _system("st2d_n8_p1_nu1e-2")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, max_iter=2)
    x, info = air.bicgstab_solve(A, H, torch.zeros(s.n, dtype=torch.float64, device="cuda"))
    assert info.status == 0 and info.iters == 0 and float(x.abs().max()) == 0.0
    x, info = air.bicgstab_solve(A, H, torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda(), rtol=1e-14)
    assert info.status == 1 and info.iters == 2 and info.relres > 1e-14
