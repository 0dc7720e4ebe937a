"""Many right-hand sides through one hierarchy (air_vcycle_multi,
air_bicgstab_solve_multi) against the single-system calls and the oracle."""
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
}
_cache = {}


def _system(name):
    if name not in _cache:
        _cache[name] = _CASES[name]()
    return _cache[name]


def _columns(s, k, seed=21):
    rng = np.random.default_rng(seed)
    B = np.empty((s.n, k))
    B[:, 0] = s.rhs
    B[:, 1:] = rng.standard_normal((s.n, k - 1))
    return B


@pytest.mark.parametrize("name", list(_CASES))
@pytest.mark.parametrize("k", [1, 5, 32])
def test_vcycle_multi_equals_single_vcycles(name, k):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100)                     # FP64 hierarchy
    B = _columns(s, k)
    X = air.vcycle_multi(H, torch.from_numpy(B).cuda()).cpu().numpy()
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    for j in range(k):
        xj = H.vcycle(torch.from_numpy(np.ascontiguousarray(B[:, j])).cuda()).cpu().numpy()
        assert np.linalg.norm(X[:, j] - xj) <= 1e-13 * np.linalg.norm(xj), j
        if j < 2:
            xo = O.vcycle(B[:, j])
            assert np.linalg.norm(X[:, j] - xo) <= 1e-10 * np.linalg.norm(xo)


def test_vcycle_multi_uses_fp64_data_of_a_low_precision_hierarchy():
    s = _system("st2d_n6_p2_nu1e-6")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H64 = air.setup(A, theta=0.25, max_coarse=100)
    H32 = air.setup(A, theta=0.25, max_coarse=100, precision=1)
    B = torch.from_numpy(_columns(s, 4)).cuda()
    assert torch.equal(air.vcycle_multi(H64, B), air.vcycle_multi(H32, B))


@pytest.mark.parametrize("name", list(_CASES))
def test_bicgstab_multi_matches_single_solves(name):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100)
    k = 6
    B = _columns(s, k)
    B[:, 3] = 0.0                                                    # a zero right-hand side converges at once
    X, infos = air.bicgstab_solve_multi(A, H, torch.from_numpy(B).cuda(), rtol=1e-12)
    X = X.cpu().numpy()
    for j in range(k):
        b = np.ascontiguousarray(B[:, j])
        r = b - oracle.spmv(s.row_ptr, s.col, s.val, X[:, j])
        if j == 3:
            assert infos[j].status == 0 and infos[j].iters == 0 and not X[:, j].any()
            continue
        x1, i1 = air.bicgstab_solve(A, H, torch.from_numpy(b).cuda(), rtol=1e-12)
        assert infos[j].status == 0 and abs(infos[j].iters - i1.iters) <= 1, (j, infos[j].iters, i1.iters)
        assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b) * (1 + 1e-6)
        x1 = x1.cpu().numpy()
        assert np.linalg.norm(X[:, j] - x1) <= 1e-9 * np.linalg.norm(x1)


def test_multi_rejects_bad_k():
    s = _system("st1d_n32_p1")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100)
    with pytest.raises(air.AirError) as e:
        air.vcycle_multi(H, torch.zeros((s.n, 33), dtype=torch.float64, device="cuda"))
    assert e.value.status == -1


@pytest.mark.parametrize("name", list(_CASES))
def test_vcycle_multi_f32_matches_single_fp32_vcycles(name):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, precision=1)
    k = 8
    B = _columns(s, k)
    X = air.vcycle_multi(H, torch.from_numpy(B).float().cuda()).double().cpu().numpy()
    for j in range(k):
        xj = H.vcycle(torch.from_numpy(np.ascontiguousarray(B[:, j])).cuda()).cpu().numpy()
        assert np.linalg.norm(X[:, j] - xj) <= 1e-5 * np.linalg.norm(xj), j


def test_bicgstab_multi_fp32_preconditioner():
    s = _system("st2d_n6_p2_nu1e-6")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, precision=1)
    k = 4
    B = _columns(s, k)
    X, infos = air.bicgstab_solve_multi(A, H, torch.from_numpy(B).cuda(), rtol=1e-10)
    X = X.cpu().numpy()
    for j in range(k):
        b = np.ascontiguousarray(B[:, j])
        _, i1 = air.bicgstab_solve(A, H, torch.from_numpy(b).cuda(), rtol=1e-10)
        assert infos[j].status == 0 and abs(infos[j].iters - i1.iters) <= 2, (j, infos[j].iters, i1.iters)
        r = b - oracle.spmv(s.row_ptr, s.col, s.val, X[:, j])
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)
