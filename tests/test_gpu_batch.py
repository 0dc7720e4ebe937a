"""Independent problems at once: air_setup_batch / air_gmres_solve_batch.

Each problem of a batch must come out exactly as from the single-problem
calls (the same kernels run, only on concurrent streams), match the oracle,
and report its own errors; concurrent setups must overlap on the GPU.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2010_11130_gb300 as air  # noqa: E402
from sthdg import assemble  # noqa: E402
from sthdg.problems import batched_problems, manufactured_2d  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    air.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


_sys = {}


def _systems():
    if "b" not in _sys:
        probs, _ = batched_problems(count=5, n_range=(3, 7))
        _sys["b"] = [assemble(p) for p in probs]
    return _sys["b"]


def _levels_equal(H1, H2):
    assert H1.levels() == H2.levels()
    for l in range(H1.levels()):
        for what in ("A.row_ptr", "A.col", "A.val"):
            assert np.array_equal(H1.export(l, what), H2.export(l, what)), (l, what)
        if H1.info(l).coarsest:
            continue
        for what in ("cf", "R.col", "R.val", "pcol"):
            assert np.array_equal(H1.export(l, what), H2.export(l, what)), (l, what)


def test_setup_batch_equals_single_setups_and_oracle():
    ss = _systems()
    As = [air.CSR.from_host(s.row_ptr, s.col, s.val) for s in ss]
    Hs, st = air.setup_batch(As, theta=0.25, max_coarse=100)
    assert st == [0] * len(ss)
    for s, A, H in zip(ss, As, Hs):
        _levels_equal(H, air.setup(A, theta=0.25, max_coarse=100))
        O = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
        assert H.levels() == len(O.levels)
        for l, OL in enumerate(O.levels):
            if OL.nc:
                assert np.array_equal(H.export(l, "cf"), OL.cf)
                assert np.array_equal(H.export(l, "R.val"), OL.R[2])


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_batch_equals_single_solves(precision):
    ss = _systems()
    As = [air.CSR.from_host(s.row_ptr, s.col, s.val) for s in ss]
    Hs, _ = air.setup_batch(As, theta=0.25, max_coarse=100, precision=precision)
    bs = [torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda() for s in ss]
    xs, infos, st = air.gmres_solve_batch(As, Hs, bs, rtol=1e-8)
    assert st == [0] * len(ss)
    for A, H, b, x, inf in zip(As, Hs, bs, xs, infos):
        x1, inf1 = air.gmres_solve(A, H, b, rtol=1e-8)
        torch.cuda.synchronize()
        assert inf.iters == inf1.iters and inf.relres == inf1.relres
        assert torch.equal(x, x1)


def test_batch_reports_each_problem_status():
    ss = _systems()[:3]
    As = [air.CSR.from_host(s.row_ptr, s.col, s.val) for s in ss]
    bad = ss[1]
    col = bad.col.copy()
    col[5] = bad.n + 7                                      # out-of-range column in problem 1 only
    As[1] = air.CSR.from_host(bad.row_ptr, col, bad.val)
    Hs, st = air.setup_batch(As, theta=0.25, max_coarse=100)
    assert st[0] == 0 and st[2] == 0 and st[1] == -2
    assert Hs[1] is None and Hs[0] is not None and Hs[2] is not None
    b = [torch.from_numpy(np.ascontiguousarray(ss[0].rhs)).cuda()] * 2
    with pytest.raises(air.AirError) as e:                 # one hierarchy twice in a solve batch
        air.gmres_solve_batch([As[0], As[0]], [Hs[0], Hs[0]], b)
    assert e.value.status == -1


def test_concurrent_setups_overlap():
    # four identical mid-size systems: the first pass of each runs on one SM, so
    # the batch takes much less than four single setups
    s = assemble(manufactured_2d(10, 2, 1e-6))
    As = [air.CSR.from_host(s.row_ptr, s.col, s.val) for _ in range(4)]
    air.setup(As[0])                                         # warm-up (module load, pools)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for A in As:
        air.setup(A)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    Hs, st = air.setup_batch(As)
    torch.cuda.synchronize()
    t_bat = time.perf_counter() - t0
    assert st == [0] * 4
    assert t_bat < 0.7 * t_seq, (t_bat, t_seq)


def test_setup_batch_distance2_equals_single_setups():
    ss = _systems()[:3]
    As = [air.CSR.from_host(s.row_ptr, s.col, s.val) for s in ss]
    Hs, st = air.setup_batch(As, theta=0.25, distance=2, max_coarse=100)
    assert st == [0] * len(ss)
    for A, H in zip(As, Hs):
        _levels_equal(H, air.setup(A, theta=0.25, distance=2, max_coarse=100))


def test_solve_batch_mixed_hierarchies_restarts_and_stops():
    # FP64, FP32 and BF16 hierarchies in one batch; GMRES(4) so that cycles end
    # and restart at different rounds; one problem stopped by max_iter and one
    # with a zero right-hand side; each must equal its single-problem solve
    ss = _systems()[:4]
    As = [air.CSR.from_host(s.row_ptr, s.col, s.val) for s in ss]
    opts = [dict(precision=0, restart=4), dict(precision=1, restart=4),
            dict(precision=2, restart=30, max_iter=3), dict(precision=1, restart=4)]
    Hs = [air.setup(A, theta=0.25, max_coarse=100, **o) for A, o in zip(As, opts)]
    bs = [torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda() for s in ss]
    bs[3] = torch.zeros_like(bs[3])
    xs, infos, st = air.gmres_solve_batch(As, Hs, bs, rtol=1e-8)
    assert st[0] == 0 and st[1] == 0 and st[3] == 0 and st[2] == 1, st
    assert infos[2].iters == 3 and infos[3].iters == 0
    assert infos[0].restarts > 1 and infos[1].restarts > 1
    for A, H, b, x, inf in zip(As, Hs, bs, xs, infos):
        x1, inf1 = air.gmres_solve(A, H, b, rtol=1e-8)
        torch.cuda.synchronize()
        assert (inf.iters, inf.restarts, inf.vcycles) == (inf1.iters, inf1.restarts, inf1.vcycles)
        assert inf.relres == inf1.relres
        assert torch.equal(x, x1)
    assert float(xs[3].abs().max()) == 0.0


def test_solve_batch_with_host_problems():
    # host CSR, right-hand sides and solutions: staged through the hierarchies'
    # device buffers, as in the single-problem host path
    ss = _systems()[:3]
    As = [air.CSR(np.ascontiguousarray(s.row_ptr, dtype=np.int64), np.ascontiguousarray(s.col, dtype=np.int32),
                  np.ascontiguousarray(s.val, dtype=np.float64), s.n) for s in ss]
    Hs = [air.setup(A, theta=0.25, max_coarse=100, precision=1) for A in As]
    bs = [torch.from_numpy(np.ascontiguousarray(s.rhs)) for s in ss]
    xs, infos, st = air.gmres_solve_batch(As, Hs, bs, rtol=1e-8)
    assert st == [0] * len(ss)
    for A, H, s, x, inf in zip(As, Hs, ss, xs, infos):
        x1, inf1 = air.gmres_solve(A, H, np.ascontiguousarray(s.rhs), rtol=1e-8)
        assert inf.iters == inf1.iters and inf.relres == inf1.relres
        assert np.array_equal(x.numpy(), x1)
