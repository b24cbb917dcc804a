"""Pins for the oracle's symbolic phase (Algorithm 1, Def. 2.3).

The oracle is checked against things other than itself:
* the path form of Def. 2.3: level(i, j) + 1 is the length of the shortest
  path i -> j in the graph of A whose intermediate vertices are all below
  min(i, j) (the fill-path characterisation of Hysom & Pothen, which the paper
  cites); computed here by breadth-first search on every pair;
* k >= n gives the structural pattern of complete LU (Sec. 2: k = infinity is
  full LU), computed by boolean Gaussian elimination;
* k = 0 keeps exactly A's pattern, patterns are nested in k, tridiagonal
  matrices never fill, and k = 1 is the closed-form union of Sec. 3.3.
"""
from collections import deque

import numpy as np
import pytest

import oracle
from paper_0803_0048_gb300 import workloads as W


def pattern_of(A):
    return {(i, int(c)) for i in range(A.n) for c in A.colind[A.rowptr[i]:A.rowptr[i + 1]]}


def path_levels(A):
    """level[i][j] by BFS over vertices < min(i, j) (None if unreachable)."""
    n = A.n
    adj = [list(A.colind[A.rowptr[i]:A.rowptr[i + 1]]) for i in range(n)]
    lev = [[None] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            lim = min(i, j)
            # shortest path with >= 1 edge from i to j, intermediates < lim
            dist = {}
            dq = deque()
            for t in adj[i]:
                if t == j:
                    dist = {j: 1}
                    break
                if t < lim and t not in dist:
                    dist[t] = 1
                    dq.append(t)
            if dist.get(j) == 1:
                lev[i][j] = 0
                continue
            found = None
            while dq and found is None:
                u = dq.popleft()
                for t in adj[u]:
                    if t == j:
                        found = dist[u] + 1
                        break
                    if t < lim and t not in dist:
                        dist[t] = dist[u] + 1
                        dq.append(t)
            lev[i][j] = None if found is None else found - 1
    return lev


def oracle_levels(A, k):
    st, bad, frp, fci, flev = oracle.symbolic(A.n, A.rowptr, A.colind, k)
    assert st in (oracle.OK, oracle.ENODIAG)
    out = {}
    for i in range(A.n):
        for p in range(frp[i], frp[i + 1]):
            out[(i, int(fci[p]))] = int(flev[p])
    return st, out


CASES = [(n, dens, seed, diag) for n, dens, seed, diag in
         [(6, 0.3, 1, True), (8, 0.25, 2, True), (10, 0.2, 3, True), (12, 0.15, 4, True),
          (14, 0.12, 5, True), (9, 0.3, 6, False), (11, 0.2, 7, False), (14, 0.2, 8, True),
          (13, 0.1, 9, False), (7, 0.5, 10, True)]]


@pytest.mark.parametrize("n,dens,seed,diag", CASES)
def test_levels_match_shortest_lower_paths(n, dens, seed, diag):
    A = W.random_sparse(n, dens, seed, diag=diag, dominance=None)
    lev = path_levels(A)
    for k in range(0, n + 1):
        st, got = oracle_levels(A, k)
        want = {(i, j): lev[i][j] for i in range(n) for j in range(n)
                if lev[i][j] is not None and lev[i][j] <= k}
        assert got == want, f"k={k}"
        has_all_diag = all((i, i) in want for i in range(n))
        assert (st == oracle.OK) == has_all_diag


def boolean_lu(mask):
    M = mask.copy()
    n = M.shape[0]
    for h in range(n):
        rows = np.nonzero(M[h + 1:, h])[0] + h + 1
        cols = np.nonzero(M[h, h + 1:])[0] + h + 1
        M[np.ix_(rows, cols)] = True
    return M


@pytest.mark.parametrize("n,dens,seed", [(20, 0.1, 11), (40, 0.05, 12), (60, 0.04, 13)])
def test_full_level_is_complete_lu_pattern(n, dens, seed):
    A = W.random_sparse(n, dens, seed)
    mask = W.csr_to_dense(A) != 0
    want = boolean_lu(mask)
    st, got = oracle_levels(A, 250)
    assert st == oracle.OK
    G = np.zeros((n, n), dtype=bool)
    for (i, j) in got:
        G[i, j] = True
    assert (G == want).all()


def test_k0_is_pattern_of_A_and_nested():
    A = W.random_sparse(80, 0.04, 21)
    st, g0 = oracle_levels(A, 0)
    assert set(g0) == pattern_of(A) and set(g0.values()) == {0}
    prev = set(g0)
    for k in range(1, 6):
        _, gk = oracle_levels(A, k)
        assert prev <= set(gk)
        # levels of entries already present do not change with k
        for key in prev:
            assert gk[key] == g0.get(key, gk[key]) or key not in g0
        prev = set(gk)


def test_tridiagonal_never_fills():
    n = 50
    main = np.arange(n)
    mask = np.zeros((n, n), dtype=bool)
    mask[main, main] = True
    mask[main[1:], main[:-1]] = True
    mask[main[:-1], main[1:]] = True
    A = W.dense_to_csr(np.where(mask, 1.0, 0.0), mask)
    for k in (0, 1, 3, 250):
        _, g = oracle_levels(A, k)
        assert set(g) == pattern_of(A)


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_k1_closed_form(seed):
    """Sec. 3.3: with k = 1 only level-0 entries cause fill, so row j's
    pattern is A_j plus {t > h : h in A_j, h < j, t in A_h}."""
    A = W.random_sparse(120, 0.03, seed)
    _, g = oracle_levels(A, 1)
    rows = [set(int(c) for c in A.colind[A.rowptr[i]:A.rowptr[i + 1]]) for i in range(A.n)]
    want = {}
    for j in range(A.n):
        for t in rows[j]:
            want[(j, t)] = 0
        for h in rows[j]:
            if h < j:
                for t in rows[h]:
                    if t > h and t not in rows[j]:
                        want[(j, t)] = 1
    assert g == want


def test_five_point_grid_fill_diagonals():
    """Saad, Iterative Methods for Sparse Linear Systems, Sec. 10.3: ILU(1)
    on the 5-point matrix adds the fill diagonals at offsets +-(N-1)
    (interior of the grid), and level(i, i+N-1) = 1."""
    N = 6
    A = W.conv_diff(N, 2, (0.0, 0.0))
    _, g = oracle_levels(A, 1)
    for i in range(A.n):
        x = i % N
        if x > 0 and i + N - 1 < A.n:
            assert g.get((i, i + N - 1)) == 1
        if x < N - 1 and i - N + 1 >= 0:
            assert g.get((i, i - N + 1)) == 1
    extra = {key for key, v in g.items() if v == 1}
    assert all(abs(j - i) == N - 1 for (i, j) in extra)


def test_bad_patterns_rejected():
    rp = np.array([0, 2, 3], dtype=np.int64)
    ci = np.array([1, 0, 1], dtype=np.int32)  # unsorted row 0
    st, bad, *_ = oracle.symbolic(2, rp, ci, 1)
    assert st == oracle.EPATTERN and bad == 0
    ci = np.array([0, 0, 1], dtype=np.int32)  # duplicate
    st, bad, *_ = oracle.symbolic(2, rp, ci, 1)
    assert st == oracle.EPATTERN and bad == 0
    ci = np.array([0, 1, 2], dtype=np.int32)  # out of range
    st, bad, *_ = oracle.symbolic(2, rp, ci, 1)
    assert st == oracle.EPATTERN and bad == 1
