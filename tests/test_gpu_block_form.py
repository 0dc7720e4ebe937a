"""The block form of the finest operator (air_options.block_size): the
relaxation sweeps and the Krylov matrix products of level 0 read one column
index per b x b facet block and the block's values as runs.  Only the storage
and the order of a row's sum change, so the FP64 V-cycle stays within 1e-10
of the oracle, the FP32 and BF16 V-cycles within their derived bounds, GMRES
within one iteration, and a matrix without that structure falls back to the
entry form."""
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


_CASES = {   # name: (system, b)
    "st1d_n32_p1": (lambda: assemble(manufactured_1d(32, 1, 1e-4)), 2),
    "st1d_n12_p2": (lambda: assemble(manufactured_1d(12, 2, 1e-3)), 3),
    "st2d_n6_p2_nu1e-6": (lambda: assemble(manufactured_2d(6, 2, 1e-6)), 6),
    "st2d_n8_p1_nu1e-2": (lambda: assemble(manufactured_2d(8, 1, 1e-2)), 3),
    "st2d_n5_p3_nu1e-5": (lambda: assemble(manufactured_2d(5, 3, 1e-5)), 10),
}
_cache = {}


def _system(name):
    if name not in _cache:
        _cache[name] = _CASES[name][0]()
    return _cache[name], _CASES[name][1]


@pytest.mark.parametrize("name", list(_CASES.keys()))
def test_block_form_vcycle_and_gmres_match_oracle(name):
    s, b = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    rng = np.random.default_rng(2)
    bs = [s.rhs, rng.standard_normal(s.n)]
    for prec, tol in ((0, 1e-10), (1, 1e-4), (2, 5e-2)):
        H = air.setup(A, theta=0.25, max_coarse=100, precision=prec, block_size=b)
        for rhs in bs:
            x = H.vcycle(torch.from_numpy(np.ascontiguousarray(rhs)).cuda())
            torch.cuda.synchronize()
            xo = O.vcycle(rhs)
            assert np.linalg.norm(x.cpu().numpy() - xo) <= tol * np.linalg.norm(xo), prec
        H.free()
    H = air.setup(A, theta=0.25, max_coarse=100, block_size=b)
    x, info = air.gmres_solve(A, H, torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda(), rtol=1e-8)
    torch.cuda.synchronize()
    xo, ito, _, oko, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-8)
    assert info.status == 0 and oko and abs(info.iters - ito) <= 1
    r = s.rhs - oracle.spmv(s.row_ptr, s.col, s.val, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(s.rhs) * (1 + 1e-6)


def test_block_form_equals_entry_form_to_rounding():
    s, b = _system("st2d_n6_p2_nu1e-6")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H0 = air.setup(A, theta=0.25, max_coarse=100)
    H1 = air.setup(A, theta=0.25, max_coarse=100, block_size=b)
    rhs = torch.from_numpy(np.random.default_rng(4).standard_normal(s.n)).cuda()
    x0, x1 = H0.vcycle(rhs), H1.vcycle(rhs)
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(x0 - x1) / torch.linalg.norm(x0)) <= 1e-13
    _, i0 = air.gmres_solve(A, H0, rhs, rtol=1e-10)
    _, i1 = air.gmres_solve(A, H1, rhs, rtol=1e-10)
    assert abs(i0.iters - i1.iters) <= 1


def test_block_form_falls_back_when_the_structure_does_not_match():
    s, b = _system("st2d_n6_p2_nu1e-6")          # blocks of 6
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    H = air.setup(A, theta=0.25, max_coarse=100, block_size=4)       # no aligned 4-blocks here
    x = H.vcycle(torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda())
    torch.cuda.synchronize()
    xo = O.vcycle(s.rhs)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)
    with pytest.raises(air.AirError):
        air.setup(A, block_size=-1)


@pytest.mark.parametrize("autotune", [0, 1])
def test_lanes_per_row_rule_and_autotuner(autotune):
    """Coarse levels (long Galerkin rows, few of them) run their sweeps and
    restriction with several lanes per row, chosen by a rule on the stored row
    width or by timing 1..32 lanes on the level's data; the V-cycle stays within
    1e-10 of the oracle either way."""
    s = assemble(manufactured_2d(12, 2, 1e-6), workers=8)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, block_size=6, autotune=autotune)
    lanes = [(H.info(l).lanes_f, H.info(l).lanes_c, H.info(l).lanes_r) for l in range(H.levels() - 1)]
    assert all(v in (1, 2, 4, 8, 16, 32) for t in lanes for v in t)
    if autotune == 0:
        assert max(max(t) for t in lanes[1:]) > 1            # some coarse level splits its rows
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    x = H.vcycle(torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda())
    torch.cuda.synchronize()
    xo = O.vcycle(s.rhs)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("relax", ["F", "FC", "FCF", "FFCFF", "A", "CAF"])
@pytest.mark.parametrize("blocked", [False, True])
def test_alternating_sweeps_match_oracle(relax, blocked):
    # Jacobi sweeps alternate between two full vectors (each launch also copies
    # the rows its point set leaves unchanged); odd and even sweep counts end in
    # the output vector, 'A' sweeps both sets from the same old vector
    s, b = _system("st2d_n6_p2_nu1e-6")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, relax=relax, omega=0.9, block_size=b if blocked else 0)
    assert H.info(0).block_size == (b if blocked else 0)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100, relax=relax, omega=0.9)
    rng = np.random.default_rng(11)
    for rhs in (s.rhs, rng.standard_normal(s.n)):
        x = H.vcycle(torch.from_numpy(np.ascontiguousarray(rhs)).cuda())
        torch.cuda.synchronize()
        xo = O.vcycle(rhs)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", ["st1d_n12_p2", "st2d_n6_p2_nu1e-6"])
def test_hierarchy_spmv_is_the_operator(name):
    # air_hierarchy_spmv: the FP64 copy of A that the Krylov solves use (block
    # form and entry form) against y = A x in float64 on the host
    s, b = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    x = np.random.default_rng(5).standard_normal(s.n)
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    y_ref = np.zeros(s.n)
    np.add.at(y_ref, rows, s.val * x[s.col])
    scale = np.zeros(s.n)
    np.add.at(scale, rows, np.abs(s.val * x[s.col]))
    for bs in (0, b):
        H = air.setup(A, theta=0.25, max_coarse=100, block_size=bs)
        y = H.spmv(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        assert np.all(np.abs(y.cpu().numpy() - y_ref) <= 1e-14 * scale + 1e-300)
