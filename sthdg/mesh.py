"""Structured all-at-once space-time simplex meshes (Section 2.2).

The space-time box is split into n^D cubes and every cube into D! simplices
(Kuhn / Freudenthal split along one main diagonal), so there are no hanging
nodes and no time levels inside the domain except the two ends, as in the
all-at-once approach.  Coordinates are ordered (t, x) for D = 2 and (t, x, y)
for D = 3; vertex ids are time-major.

Facets are numbered by their sorted global vertex tuple (lexicographic), so
both elements sharing a facet see the same canonical vertex order; the trace
basis is defined in that canonical frame.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

INTERIOR, DIRICHLET, NEUMANN = 0, 1, 2


@dataclass
class Mesh:
    D: int                       # space-time dimension (d + 1)
    n: int                       # cubes per direction
    lattice: np.ndarray          # (V, D) integer lattice coordinates
    verts: np.ndarray            # (V, D) physical coordinates (t, x[, y])
    elems: np.ndarray            # (E, D+1) vertex ids, Kuhn path order
    facets: np.ndarray           # (F, D) sorted vertex ids
    elem_facets: np.ndarray      # (E, D+1) facet opposite local vertex k
    facet_elems: np.ndarray      # (F, 2) adjacent elements (-1 if none), ascending
    facet_local: np.ndarray      # (F, 2) local facet index in those elements
    facet_kind: np.ndarray       # (F,) INTERIOR / DIRICHLET / NEUMANN
    reflect: tuple = field(default=())

    @property
    def n_elems(self) -> int:
        return self.elems.shape[0]

    @property
    def n_facets(self) -> int:
        return self.facets.shape[0]


def kuhn_paths(D: int):
    """Vertex offset paths of the D! Kuhn simplices of the unit cube."""
    paths = []
    for perm in itertools.permutations(range(D)):
        o = np.zeros((D + 1, D), dtype=np.int64)
        for k in range(D):
            o[k + 1] = o[k]
            o[k + 1, perm[k]] += 1
        paths.append(o)
    return np.stack(paths)                      # (D!, D+1, D)


def choose_reflection(D: int, a_mean) -> tuple:
    """Pick the Kuhn diagonal that keeps the mean space-time velocity off the facets.

    Interior Kuhn facets lie in planes y_i = y_j of the (possibly reflected)
    coordinates y, with normal s_i e_i - s_j e_j (s = -1 on reflected axes).
    The reflection maximising min |a_hat . normal| over those families is
    returned (time axis never reflected; ties -> first in lexicographic
    order).  With a_hat . normal = 0 on a facet and nu = 0 the facet is
    characteristic and the trace system is singular there.
    """
    ahat = np.concatenate([[1.0], np.asarray(a_mean, dtype=np.float64).reshape(-1)])
    best, best_r = -1.0, None
    for rs in itertools.product((0, 1), repeat=D - 1):
        r = (0,) + rs
        s = np.where(np.array(r) == 1, -1.0, 1.0)
        m = min(abs(s[i] * ahat[i] - s[j] * ahat[j]) / np.sqrt(2.0)
                for i in range(D) for j in range(i + 1, D))
        if m > best + 1e-14:
            best, best_r = m, r
    return best_r


def build_mesh(D: int, n: int, reflect=None, lower=None, upper=None,
               vertex_map: Optional[Callable[[np.ndarray], np.ndarray]] = None) -> Mesh:
    """Kuhn-split n^D cube mesh of the box [lower, upper] (default [0,1]^D).

    reflect: per-axis 0/1 flags choosing the split diagonal (see
    choose_reflection).  vertex_map: optional map of the (V, D) physical
    vertex array, applied after scaling (moving / deformed domains); the
    boundary classification uses the undeformed lattice.
    """
    if reflect is None:
        reflect = (0,) * D
    reflect = tuple(int(r) for r in reflect)
    lower = np.zeros(D) if lower is None else np.asarray(lower, dtype=np.float64)
    upper = np.ones(D) if upper is None else np.asarray(upper, dtype=np.float64)
    n1 = n + 1
    # vertices, time-major ids: id = ((i_t * n1) + i_x) * n1 + i_y
    lat = np.stack(np.meshgrid(*[np.arange(n1)] * D, indexing="ij"), axis=-1).reshape(-1, D)
    verts = lower + (upper - lower) * lat / n
    if vertex_map is not None:
        verts = np.asarray(vertex_map(verts.copy()), dtype=np.float64)
    strides = n1 ** np.arange(D - 1, -1, -1)
    cubes = np.stack(np.meshgrid(*[np.arange(n)] * D, indexing="ij"), axis=-1).reshape(-1, D)
    paths = kuhn_paths(D)                                # (D!, D+1, D)
    offs = paths ^ np.array(reflect, dtype=np.int64)     # reflected offsets
    # elems[c * D! + pi, k] = id(cube c + offs[pi, k])
    corner = cubes[:, None, None, :] + offs[None, :, :, :]      # (C, D!, D+1, D)
    elems = (corner * strides).sum(-1).reshape(-1, D + 1)

    E = elems.shape[0]
    V = lat.shape[0]
    # facet k of an element = its vertices without local vertex k
    fv = np.empty((E, D + 1, D), dtype=np.int64)
    for k in range(D + 1):
        fv[:, k, :] = np.delete(elems, k, axis=1)
    fv.sort(axis=-1)
    key = np.zeros((E, D + 1), dtype=np.int64)
    for m in range(D):
        key = key * V + fv[:, :, m]
    uniq, inv = np.unique(key.reshape(-1), return_inverse=True)
    F = uniq.shape[0]
    elem_facets = inv.reshape(E, D + 1)
    facets = np.empty((F, D), dtype=np.int64)
    facets[elem_facets.reshape(-1)] = fv.reshape(-1, D)

    # adjacency: stable sort of occurrences by facet id -> element order ascending
    occ = np.argsort(inv, kind="stable")
    counts = np.bincount(inv, minlength=F)
    start = np.concatenate([[0], np.cumsum(counts)[:-1]])
    facet_elems = -np.ones((F, 2), dtype=np.int64)
    facet_local = -np.ones((F, 2), dtype=np.int64)
    first = occ[start]
    facet_elems[:, 0] = first // (D + 1)
    facet_local[:, 0] = first % (D + 1)
    two = counts == 2
    second = occ[start[two] + 1]
    facet_elems[two, 1] = second // (D + 1)
    facet_local[two, 1] = second % (D + 1)
    if np.any(counts > 2):
        raise RuntimeError("non-manifold facet")

    kind = np.zeros(F, dtype=np.int8)
    bnd = ~two
    flat = lat[facets[bnd]]                              # (Fb, D, D)
    kb = np.zeros(bnd.sum(), dtype=np.int8)
    for axis in range(D):
        on = np.all(flat[:, :, axis] == 0, axis=1) | np.all(flat[:, :, axis] == n, axis=1)
        kb[on] = NEUMANN if axis == 0 else DIRICHLET
    if np.any(kb == 0):
        raise RuntimeError("unclassified boundary facet")
    kind[bnd] = kb
    return Mesh(D=D, n=n, lattice=lat, verts=verts, elems=elems, facets=facets,
                elem_facets=elem_facets, facet_elems=facet_elems, facet_local=facet_local,
                facet_kind=kind, reflect=reflect)
