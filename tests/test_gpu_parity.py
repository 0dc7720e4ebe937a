"""GPU parity of libair against the CPU oracle, through the C ABI.

Integer outputs (strength pattern, C/F splitting, coarse ids, R/P/A_c
patterns) must be bit-exact; the setup arithmetic is evaluated without
contracted multiply-adds on both sides, so R and A_c values are compared
bit for bit as well.  FP64 V-cycle output within 1e-10 (relative, 2-norm),
GMRES iteration counts within +-1.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2010_11130_gb300 as air  # noqa: E402
from sthdg import assemble  # noqa: E402
from sthdg.problems import manufactured_1d, manufactured_2d, pure_advection  # noqa: E402

VCYCLE_RTOL = 1e-10
# FP32 hierarchy: every stored value and every sweep rounds at 2^-24; over
# ~5 levels x (restriction + 3 sweeps) with |R| row sums O(10) the relative
# deviation of one V-cycle from the FP64 one stays below ~1e-4.
VCYCLE_F32_RTOL = 1e-4
# BF16 off-diagonals (unit roundoff 2^-9 ~ 2e-3 per stored value, diagonals
# and vectors FP32): the same ~10 rounded passes bound one V-cycle's relative
# deviation by ~2e-2; 5e-2 leaves room for cancellation in the coarse rows.
VCYCLE_BF16_RTOL = 5e-2


def _cases():
    return {
        "st1d_n32_p1": lambda: assemble(manufactured_1d(32, 1, 1e-4)),
        "st2d_n6_p2_nu1e-6": lambda: assemble(manufactured_2d(6, 2, 1e-6)),
        "st2d_n8_p1_nu1e-2": lambda: assemble(manufactured_2d(8, 1, 1e-2)),
        "st2d_n5_p3_nu1e-5": lambda: assemble(manufactured_2d(5, 3, 1e-5)),
    }


_cache = {}


def _system(name):
    if name not in _cache:
        _cache[name] = _cases()[name]()
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def _built():
    air.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _setup_both(s, max_coarse=100, theta=0.25, precision=0):
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=theta, max_coarse=max_coarse, precision=precision)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=theta, max_coarse=max_coarse)
    return A, H, O


@pytest.mark.parametrize("name", list(_cases().keys()))
def test_spmv_matches_oracle(name):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    x = np.random.default_rng(5).standard_normal(s.n)
    y = air.spmv(A, torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    yo = oracle.spmv(s.row_ptr, s.col, s.val, x)
    assert np.linalg.norm(y.cpu().numpy() - yo) <= 1e-13 * np.linalg.norm(yo)


@pytest.mark.parametrize("name", list(_cases().keys()))
def test_hierarchy_bit_exact(name):
    s = _system(name)
    A, H, O = _setup_both(s)
    assert H.levels() == len(O.levels)
    for l, OL in enumerate(O.levels):
        inf = H.info(l)
        assert inf.n == OL.n and inf.nnz == OL.A[1].size
        assert np.array_equal(H.export(l, "A.row_ptr"), OL.A[0])
        assert np.array_equal(H.export(l, "A.col"), OL.A[1])
        assert np.array_equal(H.export(l, "A.val"), OL.A[2]), f"A values differ on level {l}"
        if OL.nc == 0:
            assert inf.coarsest == 1
            continue
        assert np.array_equal(H.export(l, "S.row_ptr"), OL.S[0])
        assert np.array_equal(H.export(l, "S.col"), OL.S[1])
        assert np.array_equal(H.export(l, "cf"), OL.cf)
        assert np.array_equal(H.export(l, "cid"), OL.cid)
        assert np.array_equal(H.export(l, "R.row_ptr"), OL.R[0])
        assert np.array_equal(H.export(l, "R.col"), OL.R[1])
        assert np.array_equal(H.export(l, "R.val"), OL.R[2]), f"R values differ on level {l}"
        assert np.array_equal(H.export(l, "pcol"), OL.pcol)
        assert inf.n_singular == OL.n_singular


@pytest.mark.parametrize("name", list(_cases().keys()))
def test_vcycle_f64_matches_oracle(name):
    s = _system(name)
    A, H, O = _setup_both(s)
    rng = np.random.default_rng(11)
    for b in (s.rhs, rng.standard_normal(s.n)):
        x = H.vcycle(torch.from_numpy(np.ascontiguousarray(b)).cuda())
        torch.cuda.synchronize()
        xo = O.vcycle(b)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= VCYCLE_RTOL * np.linalg.norm(xo)


@pytest.mark.parametrize("name", ["st1d_n32_p1", "st2d_n6_p2_nu1e-6"])
def test_vcycle_f32_within_derived_tolerance(name):
    s = _system(name)
    A32 = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H32 = air.setup(A32, theta=0.25, max_coarse=100, precision=1)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    x = H32.vcycle(torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda())
    torch.cuda.synchronize()
    xo = O.vcycle(s.rhs)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= VCYCLE_F32_RTOL * np.linalg.norm(xo)


@pytest.mark.parametrize("name", ["st1d_n32_p1", "st2d_n6_p2_nu1e-6"])
def test_vcycle_bf16_within_derived_tolerance(name):
    s = _system(name)
    A16 = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H16 = air.setup(A16, theta=0.25, max_coarse=100, precision=2)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    x = H16.vcycle(torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda())
    torch.cuda.synchronize()
    xo = O.vcycle(s.rhs)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= VCYCLE_BF16_RTOL * np.linalg.norm(xo)


@pytest.mark.parametrize("name", ["st1d_n32_p1", "st2d_n6_p2_nu1e-6"])
def test_fgmres_bf16_hierarchy_reaches_f64_accuracy(name):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, precision=2)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.gmres_solve(A, H, b, rtol=1e-10)
    torch.cuda.synchronize()
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    xo, ito, _, _, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-10)
    assert info.status == 0 and info.relres <= 1e-10
    assert info.iters <= ito + 10
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", list(_cases().keys()))
def test_gmres_iterations_and_residual(name):
    s = _system(name)
    A, H, O = _setup_both(s)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.gmres_solve(A, H, b, rtol=1e-8)
    torch.cuda.synchronize()
    xo, ito, rro, oko, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-8)
    assert info.status == 0 and oko
    assert abs(info.iters - ito) <= 1
    xg = x.cpu().numpy()
    r = s.rhs - oracle.spmv(s.row_ptr, s.col, s.val, xg)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(s.rhs) * (1 + 1e-6)
    assert abs(info.relres - np.linalg.norm(r) / np.linalg.norm(s.rhs)) <= 1e-12


@pytest.mark.parametrize("name", ["st1d_n32_p1", "st2d_n6_p2_nu1e-6"])
def test_fgmres_f32_hierarchy_reaches_f64_accuracy(name):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, precision=1)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.gmres_solve(A, H, b, rtol=1e-10)
    torch.cuda.synchronize()
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    xo, ito, _, _, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-10)
    assert info.status == 0 and info.relres <= 1e-10
    assert info.iters <= ito + 3
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)


def test_host_buffer_solve_equals_device_solve():
    s = _system("st2d_n6_p2_nu1e-6")
    Ah = air.CSR(s.row_ptr, s.col, s.val, s.n)
    Hh = air.setup(Ah, theta=0.25, max_coarse=100)
    xh, infh = air.gmres_solve(Ah, Hh, np.ascontiguousarray(s.rhs), rtol=1e-8)
    Ad = air.CSR.from_host(s.row_ptr, s.col, s.val)
    Hd = air.setup(Ad, theta=0.25, max_coarse=100)
    xd, infd = air.gmres_solve(Ad, Hd, torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda(), rtol=1e-8)
    torch.cuda.synchronize()
    assert infh.iters == infd.iters
    assert np.allclose(xh, xd.cpu().numpy(), rtol=0, atol=1e-14 * np.abs(xh).max())


def test_exact_reduction_two_level_pure_advection_gpu():
    """nu = 0: the GPU hierarchy agrees with the oracle bit for bit on an
    upwind system whose scaled matrix is unit lower triangular (Lemma 3.1)."""
    s = assemble(pure_advection(3, 3, 1))
    A, H, O = _setup_both(s, max_coarse=50)
    for l, OL in enumerate(O.levels[:-1]):
        assert np.array_equal(H.export(l, "cf"), OL.cf)
        assert np.array_equal(H.export(l, "R.val"), OL.R[2])


def test_malformed_csr_rejected():
    s = _system("st1d_n32_p1")
    col = s.col.copy()
    col[5], col[6] = col[6], col[5]          # unsorted row
    A = air.CSR.from_host(s.row_ptr, col, s.val)
    with pytest.raises(air.AirError) as e:
        air.setup(A)
    assert e.value.status == -2
    val = s.val.copy()
    val[10] = np.nan
    with pytest.raises(air.AirError) as e:
        air.setup(air.CSR.from_host(s.row_ptr, s.col, val))
    assert e.value.status == -2


def test_unsupported_and_invalid_options():
    s = _system("st1d_n32_p1")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    with pytest.raises(air.AirError) as e:
        air.setup(A, distance=3)
    assert e.value.status == -8
    with pytest.raises(air.AirError) as e:
        air.setup(A, distance=0)
    assert e.value.status == -1
    with pytest.raises(air.AirError) as e:
        air.setup(A, relax="FXF")
    assert e.value.status == -1


def test_not_converged_reports_info():
    s = _system("st2d_n8_p1_nu1e-2")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, max_coarse=100, max_iter=3)
    x, info = air.gmres_solve(A, H, torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda(), rtol=1e-12)
    assert info.status == 1 and info.iters == 3 and info.relres > 1e-12


def test_larger_case_spans_many_tiles():
    """988k unknowns: level sizes, patterns and C/F markers bit-exact on the
    two finest levels; V-cycle within 1e-10."""
    s = assemble(manufactured_2d(24, 2, 1e-6))
    A, H, O = _setup_both(s, max_coarse=1000)
    for l in range(2):
        OL = O.levels[l]
        assert np.array_equal(H.export(l, "cf"), OL.cf)
        assert np.array_equal(H.export(l, "R.col"), OL.R[1])
        assert np.array_equal(H.export(l + 1, "A.col"), O.levels[l + 1].A[1])
        assert np.array_equal(H.export(l + 1, "A.val"), O.levels[l + 1].A[2])
    x = H.vcycle(torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda())
    torch.cuda.synchronize()
    xo = O.vcycle(s.rhs)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= VCYCLE_RTOL * np.linalg.norm(xo)
