"""GPU assembly of the space-time HDG trace system (air_hdg_*) against the
seeded host assembly of sthdg (the numpy statement of the bilinear form,
pinned by the order-(p+1) convergence, condensed-equals-full-solve and
Table 1 pulse tests), through the C ABI.

The sparsity pattern must be identical.  Values: both sides evaluate the
same quadrature sums and solve the same small element systems by LU with
partial pivoting, in different orders; the difference is rounding amplified
by the conditioning of the element matrix A_K and of the facet diagonal block
(monomial element basis, kappa up to ~1e4 for p = 3), so each row agrees to
1e-11 of its largest entry (about kappa times a few unit roundoffs).

The velocity gradient (air_hdg_velocity_gradient) is checked against
central finite differences of the loss with dense LU solves of the host
assembly on small meshes, where every element velocity can be perturbed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2010_11130_gb300 as air  # noqa: E402
from paper_2010_11130_gb300 import hdg  # noqa: E402
from sthdg import assemble  # noqa: E402
from sthdg.mesh import build_mesh  # noqa: E402
from sthdg.problems import manufactured_1d, manufactured_2d, mapped_noisy, pure_advection, rotating_pulse  # noqa: E402

ROW_RTOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    air.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _mesh_of(prob):
    return build_mesh(prob.D, prob.n, reflect=prob.reflect, lower=prob.lower, upper=prob.upper,
                      vertex_map=prob.vertex_map)


def _gpu_data(prob, mesh, hm, tab, elem_velocity=None):
    """Problem data at the GPU-computed quadrature points (evaluated on the host)."""
    xv, xf, xF = hdg.points(hm, tab)
    xv, xf, xF = xv.cpu().numpy(), xf.cpu().numpy(), xF.cpu().numpy()
    ev = prob.elem_velocity if elem_velocity is None else elem_velocity
    if ev is not None:
        vv = np.broadcast_to(ev[:, None, :], xv.shape[:2] + (prob.D - 1,))
        vf = np.broadcast_to(ev[:, None, None, :], xf.shape[:3] + (prob.D - 1,))
    else:
        vv, vf = prob.velocity(xv), prob.velocity(xf)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    alpha = 10.0 * prob.p ** 2 if prob.alpha is None else prob.alpha
    return hdg.HdgData(prob.nu, alpha, dev(vv), dev(vf), dev(prob.source(xv)), dev(prob.u_initial(xf)),
                       dev(prob.g_dirichlet(xF)))


def _row_close(rp, got, want, rtol=ROW_RTOL):
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    scale = np.zeros(n)
    np.maximum.at(scale, rows, np.abs(want))
    err = np.zeros(n)
    np.maximum.at(err, rows, np.abs(got - want))
    worst = np.max(err / np.maximum(scale, 1e-300))
    assert worst <= rtol, worst


_CASES = {
    "st1d_n8_p1": lambda: manufactured_1d(8, 1, 1e-3),
    "st1d_n6_p3": lambda: manufactured_1d(6, 3, 1e-4),
    "st2d_n3_p1_nu1e-2": lambda: manufactured_2d(3, 1, 1e-2),
    "st2d_n3_p2_rot": lambda: manufactured_2d(3, 2, 1e-6),
    "st2d_n2_p3_nu1e-5": lambda: manufactured_2d(2, 3, 1e-5),
    "adv2d_n3_p2": lambda: pure_advection(3, 3, 2),
    "pulse_n3_p2": lambda: rotating_pulse(3, 2, 1e-3),
    "mapped_noisy_n3_p2": lambda: mapped_noisy(3, 2, 1e-4),
}


@pytest.mark.parametrize("scale", [True, False])
@pytest.mark.parametrize("name", list(_CASES.keys()))
def test_assembly_matches_host(name, scale):
    prob = _CASES[name]()
    mesh = _mesh_of(prob)
    ref = assemble(prob, mesh=mesh, scale=scale, keep_diag=True)
    tab = hdg.HdgTables(prob.D, prob.p)
    hm = hdg.HdgMesh.from_mesh(mesh)
    sys_ = hdg.assemble(hm, tab, _gpu_data(prob, mesh, hm, tab), scale=scale)
    torch.cuda.synchronize()
    A = sys_.A
    assert A.n == ref.n
    assert np.array_equal(A.row_ptr.cpu().numpy(), ref.row_ptr)
    assert np.array_equal(A.col.cpu().numpy(), ref.col)
    _row_close(ref.row_ptr, A.val.cpu().numpy(), ref.val)
    rhs = sys_.rhs.cpu().numpy()
    assert np.max(np.abs(rhs - ref.rhs)) <= ROW_RTOL * max(np.max(np.abs(ref.rhs)), 1e-300)
    lam = sys_.lam_dir.cpu().numpy()
    assert np.allclose(lam, ref.lam_dirichlet, rtol=0, atol=1e-13 * max(1.0, np.abs(ref.lam_dirichlet).max()))
    dg = sys_.diag.cpu().numpy()
    assert np.max(np.abs(dg - ref.S_diag)) <= ROW_RTOL * np.max(np.abs(ref.S_diag))


def test_gpu_assembled_system_solves_like_the_host_one():
    prob = manufactured_2d(8, 2, 1e-6)
    mesh = _mesh_of(prob)
    ref = assemble(prob, mesh=mesh)
    tab = hdg.HdgTables(3, 2)
    hm = hdg.HdgMesh.from_mesh(mesh)
    sys_ = hdg.assemble(hm, tab, _gpu_data(prob, mesh, hm, tab))
    H = air.setup(sys_.A, theta=0.25, max_coarse=100)
    x, info = air.gmres_solve(sys_.A, H, sys_.rhs, rtol=1e-10)
    Ah = air.CSR.from_host(ref.row_ptr, ref.col, ref.val)
    Hh = air.setup(Ah, theta=0.25, max_coarse=100)
    xh, infoh = air.gmres_solve(Ah, Hh, torch.from_numpy(ref.rhs).cuda(), rtol=1e-10)
    torch.cuda.synchronize()
    assert info.status == 0 and abs(info.iters - infoh.iters) <= 1
    xh = xh.cpu().numpy()
    assert np.linalg.norm(x.cpu().numpy() - xh) <= 1e-8 * np.linalg.norm(xh)


def test_larger_mesh_pattern_and_values():
    """12^3 cubes x 6 tetrahedra, p = 2 (122k unknowns): many element blocks."""
    prob = manufactured_2d(12, 2, 1e-2)
    mesh = _mesh_of(prob)
    ref = assemble(prob, mesh=mesh, workers=4)
    tab = hdg.HdgTables(3, 2)
    hm = hdg.HdgMesh.from_mesh(mesh)
    sys_ = hdg.assemble(hm, tab, _gpu_data(prob, mesh, hm, tab))
    torch.cuda.synchronize()
    assert np.array_equal(sys_.A.col.cpu().numpy(), ref.col)
    _row_close(ref.row_ptr, sys_.A.val.cpu().numpy(), ref.val)


# ------------------------------------------------------------ velocity gradient
def _loss_and_grad_gpu(prob, mesh, hm, tab, target, ev):
    """L = 1/2 ||u - target||^2 over the trace unknowns, dL/d(element velocity)."""
    sys_ = hdg.assemble(hm, tab, _gpu_data(prob, mesh, hm, tab, elem_velocity=ev))
    S = air.AdjointSolver(sys_.A, rtol=1e-13, max_coarse=100)
    b = sys_.rhs.clone()
    u = S.solve(b)
    tgt = torch.from_numpy(target).cuda()
    g = u - tgt
    adj = S.solve_adjoint(g.contiguous())
    grad = hdg.velocity_gradient(hm, tab, _gpu_data(prob, mesh, hm, tab, elem_velocity=ev), sys_, u, adj)
    L = 0.5 * float((g * g).sum())
    return L, grad.cpu().numpy()


def _loss_dense(prob, mesh, ev, target):
    prob.elem_velocity = ev
    s = assemble(prob, mesh=mesh)
    import scipy.sparse as sp
    A = sp.csr_matrix((s.val, s.col, s.row_ptr), shape=(s.n, s.n)).toarray()
    u = np.linalg.solve(A, s.rhs)
    return 0.5 * float(np.sum((u - target) ** 2))


@pytest.mark.parametrize("n,p,nu", [(2, 1, 1e-4), (2, 2, 1e-2)])
def test_velocity_gradient_matches_dense_central_differences(n, p, nu):
    prob = mapped_noisy(n, p, nu)
    mesh = _mesh_of(prob)
    ev0 = prob.elem_velocity.copy()
    # target: the trace solution of the noise-free velocity (1, 0.5)
    tgt_ev = np.broadcast_to(np.array([1.0, 0.5]), ev0.shape).copy()
    prob.elem_velocity = tgt_ev
    s0 = assemble(prob, mesh=mesh)
    import scipy.sparse as sp
    target = np.linalg.solve(sp.csr_matrix((s0.val, s0.col, s0.row_ptr), shape=(s0.n, s0.n)).toarray(), s0.rhs)
    prob.elem_velocity = ev0
    tab = hdg.HdgTables(3, p)
    hm = hdg.HdgMesh.from_mesh(mesh)
    L, grad = _loss_and_grad_gpu(prob, mesh, hm, tab, target, ev0)
    assert abs(L - _loss_dense(prob, mesh, ev0, target)) <= 1e-9 * L
    h = 1e-6
    fd = np.zeros_like(ev0)
    for e in range(ev0.shape[0]):
        for m in range(2):
            ep, em = ev0.copy(), ev0.copy()
            ep[e, m] += h
            em[e, m] -= h
            fd[e, m] = (_loss_dense(prob, mesh, ep, target) - _loss_dense(prob, mesh, em, target)) / (2 * h)
    prob.elem_velocity = ev0
    # central differences: truncation O(h^2) and rounding O(eps L / h)
    assert np.max(np.abs(grad - fd)) <= 1e-5 * np.max(np.abs(fd)) + 1e-9 * L / h


def test_velocity_gradient_8cubed_sampled_central_differences():
    """The 8^3 copy of the mapped noisy-velocity workload: gradient entries of
    sampled elements against central differences of GPU-assembled, GPU-solved
    losses (h = 1e-6)."""
    prob = mapped_noisy(8, 2, 1e-4)
    mesh = _mesh_of(prob)
    ev0 = prob.elem_velocity.copy()
    tab = hdg.HdgTables(3, 2)
    hm = hdg.HdgMesh.from_mesh(mesh)
    tgt_sys = hdg.assemble(hm, tab, _gpu_data(prob, mesh, hm, tab,
                                              elem_velocity=np.broadcast_to([1.0, 0.5], ev0.shape).copy()))
    Ht = air.setup(tgt_sys.A, theta=0.25, max_coarse=100)
    target, _ = air.gmres_solve(tgt_sys.A, Ht, tgt_sys.rhs, rtol=1e-13)
    target = target.cpu().numpy()
    L, grad = _loss_and_grad_gpu(prob, mesh, hm, tab, target, ev0)

    def loss(ev):
        sys_ = hdg.assemble(hm, tab, _gpu_data(prob, mesh, hm, tab, elem_velocity=ev))
        Hs = air.setup(sys_.A, theta=0.25, max_coarse=100)
        u, inf = air.gmres_solve(sys_.A, Hs, sys_.rhs, rtol=1e-14)
        d = u.cpu().numpy() - target
        return 0.5 * float(d @ d)

    rng = np.random.default_rng(8)
    h = 1e-6
    for e in rng.choice(ev0.shape[0], size=6, replace=False):
        for m in range(2):
            ep, em = ev0.copy(), ev0.copy()
            ep[e, m] += h
            em[e, m] -= h
            fd = (loss(ep) - loss(em)) / (2 * h)
            assert abs(grad[e, m] - fd) <= 1e-4 * np.max(np.abs(grad)) + 1e-9 * L / h, (e, m, grad[e, m], fd)


# ------------------------------------------------------ block-scaled adjoint
def test_transpose_scaled_and_block_apply_match_dense():
    """D_b^{-T} A^T D_b^T (the adjoint operator with identity diagonal blocks)
    and the block-diagonal products against dense numpy."""
    import scipy.sparse as sp
    from sthdg.problems import boundary_layer
    prob = boundary_layer(3, 3, 1e-5)
    mesh = _mesh_of(prob)
    tab = hdg.HdgTables(3, 3)
    hm = hdg.HdgMesh.from_mesh(mesh)
    sys_ = hdg.assemble(hm, tab, _gpu_data(prob, mesh, hm, tab))
    A = sys_.A
    b = tab.b
    At = air.transpose_scaled(A, b, sys_.diag)
    torch.cuda.synchronize()
    n = A.n
    Ad = sp.csr_matrix((A.val.cpu().numpy(), A.col.cpu().numpy(), A.row_ptr.cpu().numpy()), shape=(n, n)).toarray()
    Dg = sys_.diag.cpu().numpy()
    Db = np.zeros((n, n))
    for k in range(n // b):
        Db[k * b:(k + 1) * b, k * b:(k + 1) * b] = Dg[k]
    want = np.linalg.inv(Db).T @ Ad.T @ Db.T
    pat = air.transpose(A)
    assert np.array_equal(At.col.cpu().numpy(), pat.col.cpu().numpy())
    in_pattern = sp.csr_matrix((np.ones(pat.nnz), pat.col.cpu().numpy(), pat.row_ptr.cpu().numpy()),
                               shape=(n, n)).toarray() != 0
    got = sp.csr_matrix((At.val.cpu().numpy(), At.col.cpu().numpy(), At.row_ptr.cpu().numpy()),
                        shape=(n, n)).toarray()
    scale = np.abs(want).max()
    assert np.max(np.abs(got - want * in_pattern)) <= 1e-11 * scale
    # what the pattern leaves out is the roundoff-level part of the diagonal blocks
    assert np.max(np.abs(want[~in_pattern])) <= 1e-11 * scale
    x = torch.randn(n, dtype=torch.float64, device="cuda")
    xh = x.cpu().numpy()
    ops = {0: Db, 1: Db.T, 2: np.linalg.inv(Db), 3: np.linalg.inv(Db).T}
    for op, M in ops.items():
        y = air.block_diag_apply(b, sys_.diag, op, x)
        torch.cuda.synchronize()
        assert np.allclose(y.cpu().numpy(), M @ xh, rtol=1e-12, atol=1e-12 * np.abs(M @ xh).max())


@pytest.mark.parametrize("n", [6, 10])
def test_block_scaled_adjoint_solve_matches_dense(n):
    """A^T lambda = g through the block-scaled similar matrix on the
    boundary-layer problem (p = 3): lambda against the dense solve, and the
    scaled form needs no more iterations than the plain transpose."""
    import scipy.sparse as sp
    from sthdg.problems import boundary_layer
    prob = boundary_layer(n, 3, 1e-5)
    mesh = _mesh_of(prob)
    tab = hdg.HdgTables(3, 3)
    hm = hdg.HdgMesh.from_mesh(mesh)
    sys_ = hdg.assemble(hm, tab, _gpu_data(prob, mesh, hm, tab))
    g = torch.randn(sys_.A.n, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    S1 = air.AdjointSolver(sys_.A, rtol=1e-11, block=(tab.b, sys_.diag), max_coarse=100)
    lam = S1.solve_adjoint(g)
    S0 = air.AdjointSolver(sys_.A, rtol=1e-11, max_coarse=100)
    lam0 = S0.solve_adjoint(g)
    torch.cuda.synchronize()
    assert S1.info_adjoint.iters <= S0.info_adjoint.iters + 2
    if n == 6:
        A = sp.csr_matrix((sys_.A.val.cpu().numpy(), sys_.A.col.cpu().numpy(), sys_.A.row_ptr.cpu().numpy()),
                          shape=(sys_.A.n, sys_.A.n)).toarray()
        ref = np.linalg.solve(A.T, g.cpu().numpy())
        assert np.linalg.norm(lam.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.linalg.norm((lam - lam0).cpu().numpy()) <= 1e-8 * np.linalg.norm(lam0.cpu().numpy())
