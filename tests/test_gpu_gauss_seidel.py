"""Forward Gauss-Seidel relaxation on the GPU (the paper's post-relaxation,
Section 4: F points, then all points) against the oracle's sequential sweeps,
through the C ABI.  The level schedule reproduces the ascending-order sweep
exactly up to the order of each row's sum, so FP64 V-cycles agree to 1e-10,
FP32 ones to the FP32 bound, and GMRES within one iteration; Jacobi over all
points ('A') and mixed strings are checked the same way."""
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


@pytest.mark.parametrize("relax,omega", [("fa", 1.0), ("fcf", 0.8), ("a", 1.0), ("Ff", 1.0), ("A", 0.7),
                                         ("FaC", 1.0)])
@pytest.mark.parametrize("name", list(_CASES.keys()))
def test_vcycle_sweeps_match_oracle(name, relax, omega):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, relax=relax, omega=omega)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100, relax=relax, omega=omega)
    rng = np.random.default_rng(3)
    for rhs in (s.rhs, rng.standard_normal(s.n)):
        x = H.vcycle(torch.from_numpy(np.ascontiguousarray(rhs)).cuda())
        torch.cuda.synchronize()
        xo = O.vcycle(rhs)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", ["st1d_n32_p1", "st2d_n6_p2_nu1e-6"])
def test_fp32_gauss_seidel_within_bound(name):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, relax="fa", precision=1, block_size=2 if "1d" in name else 6)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100, relax="fa")
    x = H.vcycle(torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda())
    torch.cuda.synchronize()
    xo = O.vcycle(s.rhs)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-4 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", list(_CASES.keys()))
def test_gmres_with_gauss_seidel_matches_oracle(name):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, relax="fa")
    x, info = air.gmres_solve(A, H, torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda(), rtol=1e-8)
    torch.cuda.synchronize()
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100, relax="fa")
    xo, ito, _, oko, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-8)
    assert info.status == 0 and oko and abs(info.iters - ito) <= 1


def test_gauss_seidel_cuts_iterations_at_16cubed():
    """2D+time n = 16, p = 2, nu = 1e-6 (291,840 unknowns): the oracle needs 27
    GMRES iterations with FCF-Jacobi and 20 with forward Gauss-Seidel; the GPU
    matches it within one."""
    s = assemble(manufactured_2d(16, 2, 1e-6), workers=8)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    its = {}
    for relax in ("FCF", "fa"):
        H = air.setup(A, theta=0.25, max_coarse=1000, relax=relax, block_size=6)
        _, info = air.gmres_solve(A, H, b, rtol=1e-8)
        its[relax] = info.iters
        H.free()
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=1000, relax="fa", copy_levels=False)
    _, ito, _, _, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-8)
    assert abs(its["fa"] - ito) <= 1 and its["fa"] < its["FCF"]


def test_gauss_seidel_options_checked():
    s = _system("st1d_n32_p1")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    with pytest.raises(air.AirError) as e:
        air.setup(A, relax="fa", precision=2)
    assert e.value.status == -8
    H = air.setup(A, relax="fa", max_coarse=100)
    B = torch.zeros((s.n, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(air.AirError) as e:
        air.vcycle_multi(H, B)
    assert e.value.status == -8
