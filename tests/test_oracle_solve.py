"""Pins for the oracle's GMRES(m), inner products and adjoint.

* Inner products: both orders lie within the standard summation error bound
  of the exactly rounded sum (math.fsum).
* An exact preconditioner (k >= n, Sec. 2: full LU) converges in one step.
* Solutions agree with dense LAPACK solves; the reported residual is the true
  residual; without preconditioning GMRES(m >= n) terminates within n steps.
* Adjoint: lambda solves A^T lambda = g (dense check), and the chain rule
  through the matrix assembly matches central finite differences.
* Mat-vec and transpose: exact on integer values against the dense product;
  the CSR transpose equals the dense transpose and, applied twice, gives the
  matrix back.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_0803_0048_gb300 import workloads as W

EPS = np.finfo(np.float64).eps


@pytest.mark.parametrize("n", [1, 7, 4096, 4097, 20000])
@pytest.mark.parametrize("mode", [oracle.DOT_SEQ, oracle.DOT_TREE])
def test_dot_within_summation_bound(n, mode):
    x = W.uniform(W.stream_key(1, "x"), np.arange(n), -1.0, 1.0)
    y = W.uniform(W.stream_key(1, "y"), np.arange(n), -1.0, 1.0)
    exact = math.fsum((x * y).tolist())
    got = oracle.dot(x, y, mode)
    bound = 1.01 * n * EPS * float(np.abs(x * y).sum()) + 1e-300
    assert abs(got - exact) <= bound


def test_tree_dot_exact_on_integers():
    # integer-valued products are summed exactly in any order
    n = 10000
    x = np.arange(n, dtype=np.float64) % 7
    y = np.arange(n, dtype=np.float64) % 5
    assert oracle.dot(x, y, oracle.DOT_TREE) == float(np.sum((np.arange(n) % 7) * (np.arange(n) % 5)))


def test_exact_preconditioner_converges_in_one_step():
    A = W.random_sparse(40, 0.1, 3)
    F = oracle.factor(A, 250)
    b = W.uniform(W.stream_key(2, "b"), np.arange(A.n), -1, 1)
    st, x, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                                       (F["rowptr"], F["colind"], F["val"]), 10, 1e-10)
    assert st == oracle.OK and it == 1


@pytest.mark.parametrize("prec", ["none", "ilu", "iilu"])
@pytest.mark.parametrize("mode", [oracle.DOT_SEQ, oracle.DOT_TREE])
@pytest.mark.parametrize("update", [oracle.UPDATE_Z, oracle.UPDATE_MVY])
def test_gmres_matches_dense_solve(prec, mode, update):
    A = W.conv_diff(12, 2, (20.0, 20.0))
    n = A.n
    b = W.uniform(W.stream_key(3, "b"), np.arange(n), -1, 1)
    F = oracle.factor(A, 1)
    if prec == "none":
        kind, Fa = oracle.PREC_NONE, None
    elif prec == "ilu":
        kind, Fa = oracle.PREC_ILU, (F["rowptr"], F["colind"], F["val"])
    else:
        g = oracle.iiluk_build(n, F["rowptr"], F["colind"], F["val"])
        kind, Fa = oracle.PREC_IILU, (F["rowptr"], F["colind"], g)
    st, x, it, rel, cyc = oracle.gmres(n, A.rowptr, A.colind, A.val, b, kind, Fa, 20, 1e-12,
                                       dotmode=mode, update=update)
    assert st == oracle.OK
    Ad = W.csr_to_dense(A)
    ref = np.linalg.solve(Ad, b)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    true_rel = np.linalg.norm(b - Ad @ x) / np.linalg.norm(b)
    assert rel <= 1e-12
    assert abs(rel - true_rel) <= 1e-3 * true_rel + 1e-15


def test_update_forms_bit_identical_without_preconditioner():
    # M = I: z_j = v_j, so x += Z y and x += M^-1 (V y) perform the same
    # operations in the same order
    A = W.conv_diff(10, 2, (20.0, 20.0))
    b = W.uniform(W.stream_key(11, "b"), np.arange(A.n), -1, 1)
    runs = [oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_NONE, None, 7, 1e-10,
                         update=u) for u in (oracle.UPDATE_Z, oracle.UPDATE_MVY)]
    assert runs[0][0] == runs[1][0] == oracle.OK and runs[0][4] > 1
    assert runs[0][2:] == runs[1][2:]
    assert np.array_equal(runs[0][1].view(np.int64), runs[1][1].view(np.int64))


@pytest.mark.parametrize("prec", ["ilu", "iilu"])
def test_update_forms_agree_over_restarts(prec):
    # With a fixed preconditioner both cycle ends give the same iterate in
    # exact arithmetic; across several restarts they agree to rounding level
    # and with the dense solve.
    A = W.conv_diff(16, 2, (20.0, 20.0))
    n = A.n
    b = W.uniform(W.stream_key(12, "b"), np.arange(n), -1, 1)
    F = oracle.factor(A, 1)
    if prec == "ilu":
        kind, Fa = oracle.PREC_ILU, (F["rowptr"], F["colind"], F["val"])
    else:
        g = oracle.iiluk_build(n, F["rowptr"], F["colind"], F["val"])
        kind, Fa = oracle.PREC_IILU, (F["rowptr"], F["colind"], g)
    out = {}
    for u in (oracle.UPDATE_Z, oracle.UPDATE_MVY):
        st, x, it, rel, cyc = oracle.gmres(n, A.rowptr, A.colind, A.val, b, kind, Fa, 6, 1e-12,
                                           update=u)
        assert st == oracle.OK and cyc >= 3
        out[u] = x
    ref = np.linalg.solve(W.csr_to_dense(A), b)
    for x in out.values():
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(out[oracle.UPDATE_Z] - out[oracle.UPDATE_MVY]) <= 1e-10 * np.linalg.norm(ref)


def test_preconditioning_reduces_iterations():
    A = W.conv_diff(24, 2, (20.0, 20.0))
    b = W.uniform(W.stream_key(4, "b"), np.arange(A.n), -1, 1)
    its = []
    for kind, k in [(oracle.PREC_NONE, None), (oracle.PREC_ILU, 0), (oracle.PREC_ILU, 2)]:
        Fa = None
        if k is not None:
            F = oracle.factor(A, k)
            Fa = (F["rowptr"], F["colind"], F["val"])
        st, x, it, rel, _ = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, kind, Fa, 30, 1e-8)
        assert st == oracle.OK
        its.append(it)
    assert its[0] > its[1] > its[2]


def test_unpreconditioned_terminates_within_n():
    A = W.random_sparse(25, 0.2, 5, dominance=0.8)
    b = W.uniform(W.stream_key(5, "b"), np.arange(A.n), -1, 1)
    st, x, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_NONE, None,
                                       A.n, 1e-10)
    assert st == oracle.OK and it <= A.n and cyc == 1


def test_nonconvergence_reported():
    A = W.conv_diff(20, 2, (20.0, 20.0))
    b = W.uniform(W.stream_key(6, "b"), np.arange(A.n), -1, 1)
    st, x, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_NONE, None,
                                       5, 1e-12, maxit=12)
    assert st == oracle.ENOCONV and it == 12 and rel > 1e-12


def test_zero_rhs():
    A = W.conv_diff(5, 2, (1.0, 1.0))
    st, x, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, np.zeros(A.n))
    assert st == oracle.OK and it == 0 and not x.any()


def test_adjoint_lambda_is_transposed_solve():
    A = W.conv_diff(10, 2, (20.0, 20.0))
    n = A.n
    F = oracle.factor(A, 2)
    b = W.uniform(W.stream_key(7, "b"), np.arange(n), -1, 1)
    st, x, *_ = oracle.gmres(n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                             (F["rowptr"], F["colind"], F["val"]), 30, 1e-13)
    g = W.uniform(W.stream_key(7, "g"), np.arange(n), -1, 1)
    st, lam, gA, it, rel = oracle.adjoint(n, A.rowptr, A.colind, A.val, F["rowptr"],
                                          F["colind"], F["val"], x, g, 30, 1e-13)
    assert st == oracle.OK
    Ad = W.csr_to_dense(A)
    ref = np.linalg.solve(Ad.T, g)
    assert np.linalg.norm(lam - ref) <= 1e-10 * np.linalg.norm(ref)
    r = np.repeat(np.arange(n), np.diff(A.rowptr))
    assert np.array_equal(gA, -(lam[r] * x[A.colind]))


def test_adjoint_gradient_matches_finite_differences():
    N = 6
    P = W.fd_pattern(N, 2)
    n = P.n
    theta0 = W.log_uniform(W.stream_key(8, "t"), np.arange(n), 0.1, 10.0)
    beta = (20.0, 20.0)
    b = W.uniform(W.stream_key(8, "b"), np.arange(n), -1, 1)
    xt = W.uniform(W.stream_key(8, "xt"), np.arange(n), -1, 1)

    def solve(theta, bb):
        v = W.fd_values(P, torch.from_numpy(theta), beta).numpy()
        F = oracle.factor(W.CSR(n, P.rowptr, P.colind, v), 2)
        st, x, *_ = oracle.gmres(n, P.rowptr, P.colind, v, bb, oracle.PREC_ILU,
                                 (F["rowptr"], F["colind"], F["val"]), 30, 1e-14)
        assert st == oracle.OK
        return v, F, x

    def loss(theta, bb):
        return float(np.sum((solve(theta, bb)[2] - xt) ** 2))

    v, F, x = solve(theta0, b)
    gx = 2.0 * (x - xt)
    st, lam, gA, *_ = oracle.adjoint(n, P.rowptr, P.colind, v, F["rowptr"], F["colind"],
                                     F["val"], x, gx, 30, 1e-14)
    th = torch.from_numpy(theta0.copy()).requires_grad_(True)
    vals = W.fd_values(P, th, beta)
    (gtheta,) = torch.autograd.grad(vals, th, grad_outputs=torch.from_numpy(gA))
    gtheta = gtheta.numpy()
    for c in [0, 7, 14, 21, 35]:
        h = 1e-6 * theta0[c]
        tp, tm = theta0.copy(), theta0.copy()
        tp[c] += h
        tm[c] -= h
        fd = (loss(tp, b) - loss(tm, b)) / (2 * h)
        assert abs(fd - gtheta[c]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gtheta).max())
    for c in [1, 17, 33]:
        h = 1e-6
        bp, bm = b.copy(), b.copy()
        bp[c] += h
        bm[c] -= h
        fd = (loss(theta0, bp) - loss(theta0, bm)) / (2 * h)
        assert abs(fd - lam[c]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(lam).max())


# --- BiCGSTAB (the paper's solver, Sec. 4) ----------------------------------

def test_bicgstab_identity_is_exact_in_half_a_step():
    # A = I: p = b, v = b, alpha = (b,b)/(b,b) = 1 exactly, s = 0: x = b bit for bit
    n = 50
    A = W.dense_to_csr(np.eye(n), np.eye(n, dtype=bool))
    b = W.uniform(W.stream_key(21, "b"), np.arange(n), -1, 1)
    st, x, it, rel, half = oracle.bicgstab(n, A.rowptr, A.colind, A.val, b)
    assert st == oracle.OK and it == 1 and half and rel == 0.0
    assert np.array_equal(x, b)


def test_bicgstab_exact_preconditioner_converges_in_one_step():
    A = W.random_sparse(40, 0.1, 3)
    F = oracle.factor(A, 250)  # complete LU: M = A up to rounding
    b = W.uniform(W.stream_key(22, "b"), np.arange(A.n), -1, 1)
    st, x, it, rel, half = oracle.bicgstab(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                                           (F["rowptr"], F["colind"], F["val"]), 1e-10)
    assert st == oracle.OK and it == 1 and half


@pytest.mark.parametrize("prec", ["none", "ilu", "iilu"])
@pytest.mark.parametrize("mode", [oracle.DOT_SEQ, oracle.DOT_TREE])
def test_bicgstab_matches_dense_solve(prec, mode):
    A = W.conv_diff(12, 2, (20.0, 20.0))
    n = A.n
    b = W.uniform(W.stream_key(23, "b"), np.arange(n), -1, 1)
    F = oracle.factor(A, 1)
    if prec == "none":
        kind, Fa = oracle.PREC_NONE, None
    elif prec == "ilu":
        kind, Fa = oracle.PREC_ILU, (F["rowptr"], F["colind"], F["val"])
    else:
        g = oracle.iiluk_build(n, F["rowptr"], F["colind"], F["val"])
        kind, Fa = oracle.PREC_IILU, (F["rowptr"], F["colind"], g)
    st, x, it, rel, half = oracle.bicgstab(n, A.rowptr, A.colind, A.val, b, kind, Fa, 1e-11,
                                           2000, mode)
    assert st == oracle.OK
    xd = np.linalg.solve(W.csr_to_dense(A), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    # the reported residual is the true one
    r = b - W.csr_to_dense(A) @ x
    assert abs(rel - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-6 * rel + 1e-15


def test_bicgstab_zero_rhs_and_nonconvergence():
    A = W.conv_diff(10, 2, (20.0, 20.0))
    st, x, it, rel, half = oracle.bicgstab(A.n, A.rowptr, A.colind, A.val, np.zeros(A.n))
    assert st == oracle.OK and it == 0 and not np.any(x)
    b = W.uniform(W.stream_key(24, "b"), np.arange(A.n), -1, 1)
    st, x, it, rel, half = oracle.bicgstab(A.n, A.rowptr, A.colind, A.val, b, rtol=1e-14,
                                           maxit=3)
    assert st == oracle.ENOCONV and it == 3


def test_spmv_exact_on_integers():
    """y = A x with small integer entries: every product and partial sum is
    exact, so the result equals the dense product exactly, whatever the
    order."""
    A = W.random_sparse(300, 0.05, 21, dominance=None)
    key = W.stream_key(21, "int")
    ival = np.floor(W.uniform(key, np.arange(A.nnz), -50, 50))
    x = np.floor(W.uniform(W.stream_key(22, "int"), np.arange(A.n), -50, 50))
    B = W.CSR(A.n, A.rowptr, A.colind, ival)
    y = oracle.spmv(A.n, B.rowptr, B.colind, B.val, x)
    assert np.array_equal(y, W.csr_to_dense(B) @ x)
    # an empty row gives +0.0
    E = W.CSR(2, np.array([0, 0, 1]), np.array([1], np.int32), np.array([3.0]))
    assert np.array_equal(oracle.spmv(2, E.rowptr, E.colind, E.val, np.array([2.0, 5.0])),
                          np.array([0.0, 15.0]))


def test_transpose_is_exact_and_involutive():
    A = W.random_sparse(200, 0.07, 23, dominance=None)
    trp, tci, tv = oracle.transpose(A.n, A.rowptr, A.colind, A.val)
    T = W.CSR(A.n, trp, tci, tv)
    assert np.array_equal(W.csr_to_dense(T), W.csr_to_dense(A).T)
    for i in range(A.n):  # rows of the transpose sorted by original row
        assert np.all(np.diff(tci[trp[i]:trp[i + 1]]) > 0)
    rrp, rci, rv = oracle.transpose(A.n, trp, tci, tv)
    assert np.array_equal(rrp, A.rowptr) and np.array_equal(rci, A.colind)
    assert np.array_equal(rv, A.val)
