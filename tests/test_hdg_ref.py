"""CPU checks of the reference-element tables of the GPU HDG assembly
(paper_2010_11130_gb300/hdg_ref.py) against what their definitions fix:
quadrature exactness on the reference simplex, the Lagrange property of the
trace basis, the canonical facet frames, and the L2 projection."""
import itertools
import math

import numpy as np
import pytest

from paper_2010_11130_gb300.hdg_ref import HdgReference, gauss_jacobi, simplex_rule


def _simplex_monomial_integral(a):
    # int over the reference simplex of prod x_k^a_k = prod a_k! / (|a| + dim)!
    return np.prod([math.factorial(k) for k in a]) / math.factorial(sum(a) + len(a))


@pytest.mark.parametrize("alpha", [0, 1, 2])
def test_gauss_jacobi_exact_to_degree_2q_minus_1(alpha):
    q = 5
    x, w = gauss_jacobi(q, alpha)
    for deg in range(2 * q):
        # int_{-1}^{1} (1-x)^alpha x^deg dx by the binomial expansion of (1-x)^alpha
        exact = sum(math.comb(alpha, j) * (-1) ** j * (1 - (-1) ** (deg + j + 1)) / (deg + j + 1)
                    for j in range(alpha + 1))
        assert abs(np.sum(w * x ** deg) - exact) <= 1e-13 * max(1.0, abs(exact))


@pytest.mark.parametrize("dim,q", [(1, 3), (2, 4), (3, 5)])
def test_simplex_rule_exactness(dim, q):
    pts, wts = simplex_rule(dim, q)
    assert len(wts) == q ** dim and np.all(wts > 0) and np.all(pts >= 0) and np.all(pts.sum(1) <= 1 + 1e-15)
    for a in itertools.product(range(2 * q), repeat=dim):
        if sum(a) > 2 * q - 1:
            continue
        got = np.sum(wts * np.prod(pts ** np.array(a), axis=1))
        assert abs(got - _simplex_monomial_integral(a)) <= 1e-14


@pytest.mark.parametrize("D,p", [(2, 1), (2, 3), (3, 2), (3, 3)])
def test_trace_basis_is_lagrange_and_frames_are_consistent(D, p):
    R = HdgReference(D, p)
    # Lagrange property at the lattice nodes, via the same construction at the nodes
    from paper_2010_11130_gb300.hdg_ref import lagrange_table
    nodes = np.array(sorted(a for a in itertools.product(range(p + 1), repeat=D - 1) if sum(a) <= p),
                     dtype=float) / p
    L = lagrange_table(nodes, p)
    assert np.allclose(L, np.eye(len(nodes)), atol=1e-12)
    assert np.allclose(R.psi.sum(1), 1.0, atol=1e-13)             # partition of unity
    # facet points lie on facet k (barycentric coordinate k is 0)
    for k in range(D + 1):
        for s in range(R.nperm):
            xi = R.xi_f[k, s]
            lam = np.hstack([1 - xi.sum(1, keepdims=True), xi])
            assert np.allclose(lam[:, k], 0.0, atol=1e-15)
    # the L2 projection reproduces a trace polynomial exactly
    rng = np.random.default_rng(0)
    c = rng.standard_normal(R.b)
    assert np.allclose(R.dir_proj @ (R.psi @ c), c, atol=1e-12)


def test_element_basis_gradients_by_finite_differences():
    R = HdgReference(3, 3)
    from paper_2010_11130_gb300.hdg_ref import monomial_table
    x = np.array([[0.2, 0.3, 0.1]])
    _, g = monomial_table(x, 3)
    h = 1e-6
    for d in range(3):
        e = np.zeros((1, 3))
        e[0, d] = h
        fd = (monomial_table(x + e, 3)[0] - monomial_table(x - e, 3)[0]) / (2 * h)
        assert np.allclose(g[0, :, d], fd[0], atol=1e-8)
