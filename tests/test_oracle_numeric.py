"""Pins for the oracle's numeric phase, sweeps and TPIILU.

* k >= n on dense column-dominant matrices: LAPACK's getrf (scipy) makes no
  row swaps there, so its L and U are the complete LU of Eq. 1.
* Tridiagonal ILU(0) is exactly the Thomas algorithm (same operations).
* On every kept position, (L~U~)_ij = a_ij up to a rounding bound (the
  defining property of the incomplete factors, Sec. 2.2).
* A diagonal matrix factors to itself.
* Sweeps solve L~U~y = p (Eq. triangleSolve).
* TPIILU (Sec. 3.5): with a full pattern Eq. inversedefine gives the exact
  inverses; on any pattern, L~(I + G_L) = I and U^(I + G_U) = I hold on the
  kept positions (they are Eq. inversedefine rearranged); a bidiagonal L
  gives beta_{i,i-1} = l_{i,i-1} exactly.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_0803_0048_gb300 import workloads as W

EPS = np.finfo(np.float64).eps


def dense_factors(n, frp, fci, fv):
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        for p in range(frp[i], frp[i + 1]):
            j = int(fci[p])
            if j < i:
                L[i, j] = fv[p]
            else:
                U[i, j] = fv[p]
    return L, U


def col_dominant_dense(n, seed):
    key = W.stream_key(seed, "test.dense")
    M = W.uniform(key, np.arange(n * n), -1.0, 1.0).reshape(n, n)
    colsum = np.abs(M).sum(axis=0) - np.abs(np.diag(M))
    M[np.arange(n), np.arange(n)] = 2.0 * colsum + 1.0
    return M


@pytest.mark.parametrize("n,seed", [(5, 1), (12, 2), (30, 3)])
def test_full_level_equals_lapack_lu(n, seed):
    M = col_dominant_dense(n, seed)
    A = W.dense_to_csr(M, np.ones_like(M, dtype=bool))
    F = oracle.factor(A, 250)
    L, U = dense_factors(n, F["rowptr"], F["colind"], F["val"])
    P, Lr, Ur = sla.lu(M)
    assert np.array_equal(P, np.eye(n)), "partial pivoting should not swap here"
    assert np.allclose(L, Lr, rtol=1e-12, atol=1e-14)
    assert np.allclose(U, Ur, rtol=1e-12, atol=1e-13 * np.abs(Ur).max())


@pytest.mark.parametrize("n,seed", [(2, 1), (17, 2), (200, 3)])
def test_tridiagonal_ilu0_is_thomas(n, seed):
    key = W.stream_key(seed, "test.tri")
    lo = W.uniform(key, np.arange(n), -1.0, 1.0)
    up = W.uniform(key, n + np.arange(n), -1.0, 1.0)
    dg = 3.0 + W.uniform(key, 2 * n + np.arange(n), 0.0, 1.0)
    M = np.diag(dg) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)
    A = W.dense_to_csr(M)
    F = oracle.factor(A, 0)
    L, U = dense_factors(n, F["rowptr"], F["colind"], F["val"])
    # Thomas: u_0 = d_0; l_i = a_i / u_{i-1}; u_i = d_i - l_i * c_{i-1}
    u = np.zeros(n)
    l = np.zeros(n)
    u[0] = dg[0]
    for i in range(1, n):
        l[i] = lo[i] / u[i - 1]
        u[i] = dg[i] - l[i] * up[i - 1]
    assert np.array_equal(np.diag(U), u)
    assert np.array_equal(np.diag(L, -1), l[1:])
    assert np.array_equal(np.diag(U, 1), up[:-1])


def kept_positions_residual(A, F):
    n = A.n
    L, U = dense_factors(n, F["rowptr"], F["colind"], F["val"])
    Ad = W.csr_to_dense(A)
    LU = L @ U
    bound = (np.abs(L) @ np.abs(U))
    worst = 0.0
    for i in range(n):
        for p in range(F["rowptr"][i], F["rowptr"][i + 1]):
            j = int(F["colind"][p])
            m = min(i, j) + 2
            err = abs(LU[i, j] - Ad[i, j])
            lim = 4 * m * EPS * bound[i, j] + 1e-300
            worst = max(worst, err / lim)
    return worst


@pytest.mark.parametrize("k", [0, 1, 2, 3])
@pytest.mark.parametrize("case", ["random", "convdiff", "nondominant"])
def test_lu_equals_a_on_kept_pattern(k, case):
    if case == "random":
        A = W.random_sparse(150, 0.03, 40 + k)
    elif case == "convdiff":
        A = W.conv_diff(9, 2, (20.0, 20.0))
    else:
        A = W.random_sparse(100, 0.04, 50 + k, dominance=0.6)
    F = oracle.factor(A, k)
    assert kept_positions_residual(A, F) <= 1.0


def test_diagonal_matrix_factors_to_itself():
    d = np.array([2.0, -3.0, 0.5, 7.0])
    A = W.dense_to_csr(np.diag(d))
    F = oracle.factor(A, 2)
    assert np.array_equal(F["val"], d)


def test_zero_pivot_and_missing_diagonal_reported():
    M = np.array([[0.0, 1.0], [1.0, 2.0]])
    A = W.dense_to_csr(M, np.ones((2, 2), dtype=bool))
    st, bad, frp, fci, _ = oracle.symbolic(2, A.rowptr, A.colind, 1)
    st, bad, _ = oracle.numeric(2, A.rowptr, A.colind, A.val, frp, fci)
    assert st == oracle.EZEROPIVOT and bad == 0
    A = W.dense_to_csr(np.array([[1.0, 1.0], [1.0, 0.0]]))
    st, bad, *_ = oracle.symbolic(2, A.rowptr, A.colind, 0)
    assert st == oracle.ENODIAG and bad == 1
    # the diagonal may enter as fill (level 1 through h = 0)
    st, bad, *_ = oracle.symbolic(2, A.rowptr, A.colind, 1)
    assert st == oracle.OK
    A = W.dense_to_csr(np.array([[1.0, np.nan], [1.0, 2.0]]))
    st, bad, frp, fci, _ = oracle.symbolic(2, A.rowptr, A.colind, 0)
    st, bad, _ = oracle.numeric(2, A.rowptr, A.colind, A.val, frp, fci)
    assert st == oracle.ENONFINITE and bad == 0


@pytest.mark.parametrize("k", [0, 2])
def test_sweeps_solve_factored_system(k):
    A = W.conv_diff(10, 2, (20.0, 20.0))
    F = oracle.factor(A, k)
    n = A.n
    L, U = dense_factors(n, F["rowptr"], F["colind"], F["val"])
    p = W.uniform(W.stream_key(7, "p"), np.arange(n), -1.0, 1.0)
    y = oracle.apply(n, F["rowptr"], F["colind"], F["val"], p)
    ref = sla.solve_triangular(U, sla.solve_triangular(L, p, lower=True, unit_diagonal=True))
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    x = oracle.lsolve(n, F["rowptr"], F["colind"], F["val"], p)
    assert np.allclose(L @ x, p, rtol=0, atol=1e-13 * np.abs(p).max() * n)
    # transposed sweeps on the explicit transpose
    trp, tci, tv = oracle.transpose(n, F["rowptr"], F["colind"], F["val"])
    yt = oracle.apply_t(n, trp, tci, tv, p)
    reft = np.linalg.solve((L @ U).T, p)
    assert np.allclose(yt, reft, rtol=1e-10, atol=1e-11 * np.abs(reft).max())


def test_full_pattern_apply_is_dense_solve():
    M = col_dominant_dense(25, 9)
    A = W.dense_to_csr(M, np.ones_like(M, dtype=bool))
    F = oracle.factor(A, 250)
    p = W.uniform(W.stream_key(8, "p"), np.arange(25), -1.0, 1.0)
    y = oracle.apply(25, F["rowptr"], F["colind"], F["val"], p)
    assert np.allclose(y, np.linalg.solve(M, p), rtol=1e-12, atol=1e-14)


def split_g(n, F, g):
    GL = np.zeros((n, n))
    GU = np.zeros((n, n))
    D = np.zeros(n)
    for i in range(n):
        for p in range(F["rowptr"][i], F["rowptr"][i + 1]):
            j = int(F["colind"][p])
            if j < i:
                GL[i, j] = g[p]
            elif j > i:
                GU[i, j] = g[p]
            else:
                D[i] = g[p]
    return GL, GU, D


def test_tpiiluk_full_pattern_is_exact_inverse():
    n = 20
    M = col_dominant_dense(n, 10)
    A = W.dense_to_csr(M, np.ones_like(M, dtype=bool))
    F = oracle.factor(A, 250)
    g = oracle.iiluk_build(n, F["rowptr"], F["colind"], F["val"])
    L, U = dense_factors(n, F["rowptr"], F["colind"], F["val"])
    GL, GU, D = split_g(n, F, g)
    assert np.array_equal(D, np.diag(U))
    I = np.eye(n)
    assert np.allclose(L @ (I + GL), I, atol=1e-13)
    Uhat = U / np.diag(U)[:, None]
    assert np.allclose(Uhat @ (I + GU), I, atol=1e-13)
    p = W.uniform(W.stream_key(9, "p"), np.arange(n), -1.0, 1.0)
    y = oracle.iiluk_apply(n, F["rowptr"], F["colind"], g, p)
    assert np.allclose(y, np.linalg.solve(M, p), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_tpiiluk_identities_on_kept_pattern(k):
    A = W.conv_diff(8, 2, (20.0, 20.0)) if k != 1 else W.random_sparse(120, 0.04, 77)
    n = A.n
    F = oracle.factor(A, k)
    g = oracle.iiluk_build(n, F["rowptr"], F["colind"], F["val"])
    L, U = dense_factors(n, F["rowptr"], F["colind"], F["val"])
    GL, GU, D = split_g(n, F, g)
    I = np.eye(n)
    RL = L @ (I + GL) - I
    Uhat = U / np.diag(U)[:, None]
    RU = Uhat @ (I + GU) - I
    BL = np.abs(L) @ (I + np.abs(GL))
    BU = np.abs(Uhat) @ (I + np.abs(GU))
    for i in range(n):
        for p in range(F["rowptr"][i], F["rowptr"][i + 1]):
            j = int(F["colind"][p])
            m = abs(i - j) + 2
            if j < i:
                assert abs(RL[i, j]) <= 4 * m * EPS * BL[i, j]
            elif j > i:
                assert abs(RU[i, j]) <= 4 * m * EPS * BU[i, j]


def test_tpiiluk_bidiagonal_is_exact_copy():
    n = 30
    key = W.stream_key(12, "bi")
    M = (np.diag(4.0 + W.uniform(key, np.arange(n), 0, 1))
         + np.diag(W.uniform(key, n + np.arange(n - 1), -1, 1), -1)
         + np.diag(W.uniform(key, 2 * n + np.arange(n - 1), -1, 1), 1))
    A = W.dense_to_csr(M)
    F = oracle.factor(A, 0)
    g = oracle.iiluk_build(n, F["rowptr"], F["colind"], F["val"])
    L, U = dense_factors(n, F["rowptr"], F["colind"], F["val"])
    GL, GU, D = split_g(n, F, g)
    assert np.array_equal(np.diag(GL, -1), -np.diag(L, -1))
    assert np.array_equal(np.diag(GU, 1), -(np.diag(U, 1) / np.diag(U)[:-1]))
