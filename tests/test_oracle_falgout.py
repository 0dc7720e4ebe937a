"""Pins of the oracle's Falgout-style splitting (Section 4 names Falgout
coarsening; the reading, stated in air_oracle.c: the first pass in each block
of consecutive points on the strength graph restricted to the block, then
rounds of a parallel independent set on the interface points left F without a
strong C point).

* one block covering the level reproduces the first pass bit for bit;
* on random graphs of at most 12 points with blocks of 2 to 6 points, the
  splitting equals a brute-force statement of the definition written here
  (its local passes by the O(n^2) first pass, its interface rounds by sets);
* the weights' hash is SplitMix64: its first outputs for seed 0 are the
  published reference values 0xe220a8397b1dcdaf and 0x6e789e6aa1b965f4;
* every point left F has a strong C point or no strong connection at all
  across blocks after the rounds, on a trace system.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from sthdg import assemble
from sthdg.problems import manufactured_2d

MASK = (1 << 64) - 1


def _splitmix64(x):
    z = (x + 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def test_hash_is_splitmix64():
    assert _splitmix64(0) == 0xE220A8397B1DCDAF
    assert _splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4     # second output from seed 0
    for x in (0, 1, 7, 12345, 2 ** 40 + 3):
        assert oracle.hash_frac(x) == (_splitmix64(x) >> 11) / 2.0 ** 53


def _dense_csr(M):
    S = sp.csr_matrix(M)
    S.sort_indices()
    return S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64)


def _first_pass(S):
    """The first pass from its definition (O(n^2) scans)."""
    n = len(S)
    ST = [[i for i in range(n) if j in S[i]] for j in range(n)]
    lam = [len(ST[i]) for i in range(n)]
    state = ["F" if not S[i] and not ST[i] else "U" for i in range(n)]
    while True:
        cand = [i for i in range(n) if state[i] == "U"]
        if not cand:
            break
        best = max(cand, key=lambda i: (lam[i], -i))
        if lam[best] == 0:
            break
        state[best] = "C"
        for j in ST[best]:
            if state[j] == "U":
                state[j] = "F"
                for k in S[j]:
                    if state[k] == "U":
                        lam[k] += 1
        for k in S[best]:
            if state[k] == "U":
                lam[k] -= 1
    return [1 if s == "C" else 0 for s in state]


def _falgout(S, block):
    n = len(S)
    ST = [[i for i in range(n) if j in S[i]] for j in range(n)]
    cf = [0] * n
    for lo in range(0, n, block):
        hi = min(lo + block, n)
        local = [[k - lo for k in S[i] if lo <= k < hi] for i in range(lo, hi)]
        cf[lo:hi] = _first_pass(local)

    def has_c(i):
        return any(cf[k] == 1 for k in S[i])

    U = {i for i in range(n) if cf[i] == 0 and S[i] and not has_c(i)
         and any(k // block != i // block for k in S[i] + ST[i])}
    w = {i: len(ST[i]) + oracle.hash_frac(i) for i in range(n)}
    while U:
        sel = {i for i in U
               if not any(j in U and (w[j] > w[i] or (w[j] == w[i] and j < i)) for j in set(S[i]) | set(ST[i]))}
        assert sel
        for i in sel:
            cf[i] = 1
        U = {i for i in U - sel if not has_c(i)}
    return np.array(cf, dtype=np.int8)


@pytest.mark.parametrize("seed", range(150))
def test_falgout_matches_definition_on_small_graphs(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(4, 13))
    block = int(rng.integers(1, 7))        # one-point blocks: every connection is an interface
    M = np.eye(n) * 4.0
    mask = rng.random((n, n)) < (0.3 if seed % 2 else 0.15)
    np.fill_diagonal(mask, False)
    M[mask] = -rng.choice([1.0, 1.0, 2.0], size=mask.sum())
    H = oracle.setup(*_dense_csr(M), theta=0.25, max_coarse=0, max_levels=2, falgout_block=block)
    L = H.levels[0]
    if L.S is None:               # the level did not coarsen: nothing to compare
        return
    rp, ci = L.S
    S = [list(ci[rp[i]:rp[i + 1]]) for i in range(n)]
    assert np.array_equal(L.cf, _falgout(S, block))


def test_one_block_is_the_first_pass():
    s = assemble(manufactured_2d(4, 2, 1e-4))
    H0 = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100)
    H1 = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100, falgout_block=s.n)
    assert len(H0.levels) == len(H1.levels)
    for a, b in zip(H0.levels, H1.levels):
        assert (a.cf is None) == (b.cf is None)
        if a.cf is not None:
            assert np.array_equal(a.cf, b.cf)
            assert np.array_equal(a.R[2], b.R[2])


@pytest.mark.parametrize("block", [1024, 2048])
def test_falgout_leaves_no_uncovered_interface_point(block):
    s = assemble(manufactured_2d(5, 2, 1e-4))
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, max_coarse=100, falgout_block=block)
    for L in H.levels[:-1]:
        rp, ci = L.S
        ST = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(L.n, L.n)).T.tocsr()
        for i in range(L.n):
            Si = ci[rp[i]:rp[i + 1]]
            if L.cf[i] == 1 or len(Si) == 0 or np.any(L.cf[Si] == 1):
                continue
            nb = np.concatenate([Si, ST.indices[ST.indptr[i]:ST.indptr[i + 1]]])
            assert np.all(nb // block == i // block), i      # only points without cross-block links stay so


def test_interface_rounds_compare_both_directions():
    """One-point blocks (every connection crosses blocks) on a 6-point graph
    where a point must wait for a heavier point that depends on it (in S^T_i,
    not in S_i): comparing only S_i would leave point 0 F."""
    S = [[3, 5], [], [4, 5], [1], [0], [4]]
    M = np.eye(6) * 4.0
    for i, row in enumerate(S):
        M[i, row] = -1.0
    H = oracle.setup(*_dense_csr(M), theta=0.25, max_coarse=0, max_levels=2, falgout_block=1)
    assert list(H.levels[0].cf) == [1, 0, 0, 1, 1, 0] == list(_falgout(S, 1))
