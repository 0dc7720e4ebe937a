"""Solver variants of the paper on the GPU against the oracle.

* The strength pair (Section 4): coarsening at 0.2, R at 0.3, selected by
  air_options.theta_r; hierarchy bit for bit, solve within one iteration.
* The block-scaling ablation (Section 5.4, "No Block Inv"): the same setup on
  the unscaled condensed matrix S; hierarchy bit for bit and the same lack of
  convergence.
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
    "st2d_n5_p3_nu1e-5": lambda: assemble(manufactured_2d(5, 3, 1e-5)),
}


@pytest.mark.parametrize("name", list(_CASES))
def test_theta_pair_hierarchy_bit_exact_and_solve(name):
    s = _CASES[name]()
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.2, max_coarse=100, theta_r=0.3)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.2, theta_r=0.3, max_coarse=100)
    H1 = air.setup(A, theta=0.2, max_coarse=100)
    assert H.levels() == len(O.levels)
    for l, OL in enumerate(O.levels):
        assert np.array_equal(H.export(l, "A.val"), OL.A[2]), l
        if OL.nc == 0:
            continue
        assert np.array_equal(H.export(l, "S.col"), OL.S[1])      # the coarsening graph is exported
        assert np.array_equal(H.export(l, "cf"), OL.cf)
        assert np.array_equal(H.export(l, "R.row_ptr"), OL.R[0])
        assert np.array_equal(H.export(l, "R.col"), OL.R[1])
        assert np.array_equal(H.export(l, "R.val"), OL.R[2])
        assert np.array_equal(H.export(l, "pcol"), OL.pcol)
    if name.startswith("st2d"):          # (in 1D+time every strong entry clears both thresholds)
        assert not np.array_equal(H.export(0, "R.row_ptr"), H1.export(0, "R.row_ptr"))
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.gmres_solve(A, H, b, rtol=1e-8)
    _, ito, _, oko, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-8)
    assert info.status == 0 and oko and abs(info.iters - ito) <= 1


def test_unscaled_system_hierarchy_bit_exact_and_same_stall():
    s = assemble(manufactured_2d(4, 2, 1e-6), scale=False)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, max_iter=30)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    assert H.levels() == len(O.levels)
    for l, OL in enumerate(O.levels):
        assert np.array_equal(H.export(l, "A.val"), OL.A[2]), l
        if OL.nc:
            assert np.array_equal(H.export(l, "cf"), OL.cf)
            assert np.array_equal(H.export(l, "R.val"), OL.R[2])
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.gmres_solve(A, H, b, rtol=1e-8)
    _, ito, rro, oko, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-8, max_iter=30)
    assert info.status == 1 and not oko and info.iters == ito == 30
    assert abs(info.relres - rro) <= 1e-6 * rro
