"""Seeded synthetic space-time problems.

Each function returns a sthdg.assemble.Problem.  Coordinates are (t, x) or
(t, x, y).  The workloads follow the kinds of test problem of Section 5:
manufactured smooth solutions for convergence, the rotating Gaussian pulse of
Section 5.1 on its deforming domain, and the 2D+time rotating / constant flows
used for solver timing.  No external data is read.
"""
from __future__ import annotations

import numpy as np

from .assemble import Problem
from .mesh import choose_reflection

PI = np.pi


def manufactured_1d(n: int = 32, p: int = 1, nu: float = 1e-4, a: float = 1.0) -> Problem:
    """1D+time on [0,1]^2, u = sin(2 pi x) exp(-t), constant velocity a."""
    def u(X):
        return np.sin(2 * PI * X[..., 1]) * np.exp(-X[..., 0])

    def f(X):
        t, x = X[..., 0], X[..., 1]
        e = np.exp(-t)
        return (-np.sin(2 * PI * x) * e + a * 2 * PI * np.cos(2 * PI * x) * e
                + nu * 4 * PI * PI * np.sin(2 * PI * x) * e)

    return Problem(D=2, n=n, p=p, nu=nu,
                   velocity=lambda X: np.full(X.shape[:-1] + (1,), a),
                   source=f, g_dirichlet=u, u_initial=u, exact=u,
                   reflect=choose_reflection(2, [a]), name=f"mms1d_n{n}_p{p}",
                   spec=("manufactured_1d", dict(n=n, p=p, nu=nu, a=a)))


def manufactured_2d(n: int = 48, p: int = 2, nu: float = 1e-6, velocity: str = "rotating",
                    a_const=(0.7, 0.3)) -> Problem:
    """2D+time on [0,1]^3, u = sin(pi x) sin(pi y) cos(2 pi t).

    velocity "rotating": a = (-(y - 1/2), x - 1/2); "constant": a = a_const.
    """
    def u(X):
        t, x, y = X[..., 0], X[..., 1], X[..., 2]
        return np.sin(PI * x) * np.sin(PI * y) * np.cos(2 * PI * t)

    if velocity == "rotating":
        def vel(X):
            return np.stack([-(X[..., 2] - 0.5), X[..., 1] - 0.5], axis=-1)
        amean = [0.0, 0.0]
    else:
        ac = np.asarray(a_const, dtype=np.float64)

        def vel(X):
            return np.broadcast_to(ac, X.shape[:-1] + (2,)).copy()
        amean = ac

    def f(X):
        t, x, y = X[..., 0], X[..., 1], X[..., 2]
        sx, cx = np.sin(PI * x), np.cos(PI * x)
        sy, cy = np.sin(PI * y), np.cos(PI * y)
        ct, st = np.cos(2 * PI * t), np.sin(2 * PI * t)
        a = vel(X)
        ut = -2 * PI * sx * sy * st
        ux = PI * cx * sy * ct
        uy = PI * sx * cy * ct
        lap = -2 * PI * PI * sx * sy * ct
        return ut + a[..., 0] * ux + a[..., 1] * uy - nu * lap

    return Problem(D=3, n=n, p=p, nu=nu, velocity=vel, source=f, g_dirichlet=u,
                   u_initial=u, exact=u, reflect=choose_reflection(3, amean),
                   name=f"mms2d_{velocity}_n{n}_p{p}",
                   spec=("manufactured_2d", dict(n=n, p=p, nu=nu, velocity=velocity,
                                                 a_const=tuple(np.asarray(a_const, dtype=float)))))


def pure_advection(D: int, n: int, p: int, a=None) -> Problem:
    """nu = 0, constant velocity, smooth inflow data: the hyperbolic limit.

    With a facet-free mean velocity (choose_reflection) the element graph is
    acyclic, so the block-scaled trace matrix is unit lower triangular in a
    topological facet order (Lemma 3.1).
    """
    if a is None:
        a = [0.6] if D == 2 else [0.7, 0.3]
    a = np.asarray(a, dtype=np.float64)

    def u(X):
        s = np.zeros(X.shape[:-1])
        for k in range(1, D):
            s = s + (X[..., k] - a[k - 1] * X[..., 0])
        return np.sin(2.0 * s) + 0.5

    return Problem(D=D, n=n, p=p, nu=0.0,
                   velocity=lambda X: np.broadcast_to(a, X.shape[:-1] + (D - 1,)).copy(),
                   source=lambda X: np.zeros(X.shape[:-1]), g_dirichlet=u, u_initial=u,
                   exact=u, reflect=choose_reflection(D, a), name=f"adv{D}d_n{n}_p{p}",
                   spec=("pure_advection", dict(D=D, n=n, p=p, a=tuple(a.tolist()))))


def rotating_pulse(n: int, p: int, nu: float, A: float = 0.1) -> Problem:
    """Rotating Gaussian pulse on a time-dependent domain (Section 5.1).

    a = (-4 x2, 4 x1), f = 0, sigma = 0.1, centre (-0.2, 0.1), T = 1; the
    uniform mesh of [0,1] x [-1/2,1/2]^2 is deformed by
    x_i = x_i^u + A (1/2 - x_i^u) sin(2 pi (1/2 - x_i^* + t)), x^* = (x2^u, x1^u).
    """
    sig, xc, yc = 0.1, -0.2, 0.1

    def u(X):
        t, x1, x2 = X[..., 0], X[..., 1], X[..., 2]
        xt = x1 * np.cos(4 * t) + x2 * np.sin(4 * t)
        yt = -x1 * np.sin(4 * t) + x2 * np.cos(4 * t)
        den = 2 * sig ** 2 + 4 * nu * t
        return sig ** 2 / (sig ** 2 + 2 * nu * t) * np.exp(-((xt - xc) ** 2 + (yt - yc) ** 2) / den)

    def vmap(V):
        t, xu, yu = V[:, 0].copy(), V[:, 1].copy(), V[:, 2].copy()
        V[:, 1] = xu + A * (0.5 - xu) * np.sin(2 * PI * (0.5 - yu + t))
        V[:, 2] = yu + A * (0.5 - yu) * np.sin(2 * PI * (0.5 - xu + t))
        return V

    return Problem(D=3, n=n, p=p, nu=nu,
                   velocity=lambda X: np.stack([-4 * X[..., 2], 4 * X[..., 1]], axis=-1),
                   source=lambda X: np.zeros(X.shape[:-1]), g_dirichlet=u, u_initial=u,
                   exact=u, reflect=(0, 0, 0), lower=(0.0, -0.5, -0.5), upper=(1.0, 0.5, 0.5),
                   vertex_map=vmap, name=f"pulse_n{n}_p{p}",
                   spec=("rotating_pulse", dict(n=n, p=p, nu=nu, A=A)))


def mapped_noisy(n: int = 40, p: int = 2, nu: float = 1e-4, seed: int = 4) -> Problem:
    """Time-dependent mapped domain with a noisy piecewise-constant velocity.

    The uniform mesh of [0,1]^3 (t, x, y) is deformed by
    x' = x + 0.05 sin(2 pi t) sin(pi x) sin(pi y), y' likewise (the same
    displacement); the boundary of the space-time cube stays in place.  Each
    element e gets the constant velocity (1, 0.5) + 0.1 N(0, 1) (two draws per
    element, in element order, from numpy.random.default_rng(seed)).  Initial
    and inflow data are u = sin(pi x) sin(pi y) cos(2 pi t); the source is the
    one that makes u exact for the mean velocity (1, 0.5), so u solves the
    problem only approximately.
    """
    from .mesh import build_mesh
    base = manufactured_2d(n=n, p=p, nu=nu, velocity="constant", a_const=(1.0, 0.5))

    def vmap(V):
        t, x, y = V[:, 0].copy(), V[:, 1].copy(), V[:, 2].copy()
        d = 0.05 * np.sin(2 * PI * t) * np.sin(PI * x) * np.sin(PI * y)
        V[:, 1] = x + d
        V[:, 2] = y + d
        return V

    E = build_mesh(3, n, reflect=base.reflect).n_elems
    rng = np.random.default_rng(seed)
    ev = np.array([1.0, 0.5]) + 0.1 * rng.standard_normal((E, 2))
    return Problem(D=3, n=n, p=p, nu=nu, velocity=base.velocity, source=base.source,
                   g_dirichlet=base.g_dirichlet, u_initial=base.u_initial, exact=None,
                   reflect=base.reflect, vertex_map=vmap, elem_velocity=ev,
                   name=f"mapped_noisy_n{n}_p{p}", spec=None)


def boundary_layer(n: int = 56, p: int = 3, nu: float = 1e-5) -> Problem:
    """2D+time on [0,1]^3 with a shear layer across x = 1/2 and a Gaussian pulse.

    Velocity a = (1, 0.5 tanh(20 (x - 1/2))), f = 0, zero Dirichlet data on the
    spatial boundary, initial data u0 = exp(-200 ((x - 0.3)^2 + (y - 0.3)^2))
    imposed through the inflow flux on t = 0.  No closed-form solution.  The
    Kuhn diagonal is chosen for the mean velocity (1, 0).
    """
    def u0(X):
        x, y = X[..., 1], X[..., 2]
        return np.exp(-200.0 * ((x - 0.3) ** 2 + (y - 0.3) ** 2))

    def vel(X):
        x = X[..., 1]
        return np.stack([np.ones_like(x), 0.5 * np.tanh(20.0 * (x - 0.5))], axis=-1)

    return Problem(D=3, n=n, p=p, nu=nu, velocity=vel, source=lambda X: np.zeros(X.shape[:-1]),
                   g_dirichlet=lambda X: np.zeros(X.shape[:-1]), u_initial=u0, exact=None,
                   reflect=choose_reflection(3, [1.0, 0.0]), name=f"layer_n{n}_p{p}",
                   spec=("boundary_layer", dict(n=n, p=p, nu=nu)))


def batched_problems(count: int = 16, n_range=(16, 48), seed: int = 2010_11130):
    """Independent 2D+time problems of uneven size for batched solves.

    From numpy.random.default_rng(seed), per problem in order: n uniform on the
    integers of n_range (inclusive), p uniform on {1, 2}, phi uniform on
    [0, 2 pi), log10(nu) uniform on [-6, -2].  Velocity a = (cos phi, sin phi),
    manufactured solution and source as manufactured_2d.  Returns the problems
    and the generator (its next draws belong to the caller, e.g. extra
    right-hand sides).
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        p = int(rng.integers(1, 3))
        phi = float(rng.uniform(0.0, 2.0 * PI))
        nu = float(10.0 ** rng.uniform(-6.0, -2.0))
        out.append(manufactured_2d(n=n, p=p, nu=nu, velocity="constant", a_const=(np.cos(phi), np.sin(phi))))
    return out, rng


def make(spec) -> Problem:
    """Rebuild a problem from its (factory name, kwargs) spec."""
    name, kw = spec
    return {"manufactured_1d": manufactured_1d, "manufactured_2d": manufactured_2d,
            "pure_advection": pure_advection, "rotating_pulse": rotating_pulse,
            "boundary_layer": boundary_layer}[name](**kw)


def workload(name: str, **kw) -> Problem:
    """Named synthetic workloads.

    'st1d_n32_p1'  : 1D+time, 32x32 squares x 2 triangles, p=1, a_hat=(1,1), nu=1e-4,
                     u = sin(2 pi x) e^{-t}  (6,144 unknowns)
    'st2d_n48_p2'  : 2D+time, 48^3 cubes x 6 tetrahedra, p=2, rotating a, nu=1e-6 (or
                     nu=1e-2), u = sin(pi x) sin(pi y) cos(2 pi t)  (7,934,976 unknowns)
    Smaller 2D+time cases of the same family take n and p keywords.
    """
    if name == "st1d_n32_p1":
        return manufactured_1d(n=32, p=1, nu=kw.get("nu", 1e-4))
    if name == "st2d":
        return manufactured_2d(n=kw.get("n", 48), p=kw.get("p", 2), nu=kw.get("nu", 1e-6))
    raise KeyError(name)
