"""Inputs: the 27-point Poisson matrix (Sec. 4's 3D 27-point central
differencing) against closed forms, and the TPILU(k) solve policy of the
oracle (Sec. 1: TPIILU first, ILU(k) when it does not converge) against the
plain solves it is made of."""
import numpy as np
import pytest

import oracle
from paper_0803_0048_gb300 import workloads as W


@pytest.mark.parametrize("N", [1, 2, 5, 9])
def test_poisson27_structure(N):
    A = W.poisson27(N)
    # each dimension contributes 3N - 2 valid (point, offset) pairs
    assert A.n == N ** 3 and A.nnz == (3 * N - 2) ** 3
    D = W.csr_to_dense(A)
    assert np.array_equal(D, D.T)
    assert np.all(np.diag(D) == 26.0)
    assert set(np.unique(D[D != 26.0])) <= {0.0, -1.0}
    for i in range(A.n):
        cols = A.colind[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
    if N >= 3:  # an interior point sees all 26 neighbours: its row sums to zero
        c = (N // 2) * (1 + N + N * N)
        assert D[c].sum() == 0.0 and np.count_nonzero(D[c]) == 27


def test_oracle_tpilu_policy_branches():
    Pb = W.poisson27_problem(6, k=0)
    A = Pb.A
    F = oracle.factor(A, 0)
    Ft = (F["rowptr"], F["colind"], F["val"])
    g = oracle.iiluk_build(A.n, *Ft)
    for solver in ("gmres", "bicgstab"):
        # generous budget: TPIILU converges and its result is returned as is
        st, x, it, rel, used = oracle.tpilu(A.n, A.rowptr, A.colind, A.val, Pb.b, Ft, g, solver,
                                            30, 1e-8, 500, 500)
        assert st == oracle.OK and used == "iilu"
        if solver == "gmres":
            ref = oracle.gmres(A.n, A.rowptr, A.colind, A.val, Pb.b, oracle.PREC_IILU,
                               (Ft[0], Ft[1], g), 30, 1e-8, 500)
        else:
            ref = oracle.bicgstab(A.n, A.rowptr, A.colind, A.val, Pb.b, oracle.PREC_IILU,
                                  (Ft[0], Ft[1], g), 1e-8, 500)
        assert np.array_equal(x, ref[1]) and it == ref[2]
        # one iteration cannot reach 1e-8: the policy reverts to ILU(k) from x0 = 0
        st, x, it, rel, used = oracle.tpilu(A.n, A.rowptr, A.colind, A.val, Pb.b, Ft, g, solver,
                                            30, 1e-8, 1, 500)
        assert st == oracle.OK and used == "ilu"
        if solver == "gmres":
            ref = oracle.gmres(A.n, A.rowptr, A.colind, A.val, Pb.b, oracle.PREC_ILU, Ft, 30,
                               1e-8, 500)
        else:
            ref = oracle.bicgstab(A.n, A.rowptr, A.colind, A.val, Pb.b, oracle.PREC_ILU, Ft,
                                  1e-8, 500)
        assert np.array_equal(x, ref[1]) and it == ref[2]
