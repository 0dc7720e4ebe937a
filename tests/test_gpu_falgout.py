"""Falgout-style splitting on the GPU against the oracle, through the C ABI:
the first pass in every block of consecutive points at once (one warp per
block), then the interface rounds.  The C/F splitting and everything built
on it must be bit-exact; GMRES within one iteration."""
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


def _compare(H, O, levels=None):
    assert H.levels() == len(O.levels)
    for l, OL in enumerate(O.levels[:levels]):
        assert np.array_equal(H.export(l, "A.col"), OL.A[1])
        assert np.array_equal(H.export(l, "A.val"), OL.A[2]), l
        if OL.nc == 0:
            continue
        assert np.array_equal(H.export(l, "cf"), OL.cf), l
        assert np.array_equal(H.export(l, "R.col"), OL.R[1])
        assert np.array_equal(H.export(l, "R.val"), OL.R[2])
        assert np.array_equal(H.export(l, "pcol"), OL.pcol)


@pytest.mark.parametrize("block", [1024, 2048, 8192])
@pytest.mark.parametrize("name", list(_CASES.keys()))
def test_falgout_hierarchy_bit_exact(name, block):
    s = _system(name)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=100, falgout_block=block)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100, falgout_block=block)
    _compare(H, O)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    x, info = air.gmres_solve(A, H, b, rtol=1e-8)
    torch.cuda.synchronize()
    xo, ito, _, oko, _ = oracle.gmres(s.row_ptr, s.col, s.val, O, s.rhs, rtol=1e-8)
    assert info.status == 0 and oko and abs(info.iters - ito) <= 1


def test_falgout_larger_case_bit_exact():
    """988k unknowns, blocks of 8192 points: 121 blocks at once on level 0."""
    s = assemble(manufactured_2d(24, 2, 1e-6), workers=8)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    H = air.setup(A, theta=0.25, max_coarse=1000, falgout_block=8192)
    O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=1000, falgout_block=8192)
    _compare(H, O, levels=3)


def test_falgout_option_checked():
    s = _system("st1d_n32_p1")
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    for bad in (1000, 16384, -1024):
        with pytest.raises(air.AirError) as e:
            air.setup(A, falgout_block=bad)
        assert e.value.status == -1
