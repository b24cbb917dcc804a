"""iluk_factor runs the numeric phase beside the symbolic one in one launch
(k >= 2) and must give exactly what iluk_symbolic followed by iluk_numeric
gives: the same pattern and levels, the same factor values bit for bit
(checked against the oracle and against the two separate calls), and the
same preconditioner applications, although its sweeps walk index orders
instead of level orders.  k <= 1 and rows too long for the combined launch
take the two calls; errors are reported as the two calls report them.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0803_0048_gb300 as P
from paper_0803_0048_gb300 import _lib as L
from paper_0803_0048_gb300 import workloads as W

from gpu_helpers import assert_bits_equal, small_cases, to_dev, vec

pytestmark = pytest.mark.gpu

CASES = small_cases()
IDS = [c[0] for c in CASES]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("name,A,k", CASES, ids=IDS)
def test_factor_equals_oracle(name, A, k):
    rp, ci, av = to_dev(A)
    S, F = P.factor(rp, ci, av, k)
    ref = oracle.factor(A, k)
    grp, gci, glev, gdg = [t.cpu().numpy() for t in S.pattern()]
    assert np.array_equal(grp, ref["rowptr"]) and np.array_equal(gci, ref["colind"])
    assert np.array_equal(glev, ref["level"])
    assert_bits_equal(F.values(), ref["val"], "factor values")
    p, pd = vec(17, A.n)
    y = F.apply(pd)
    assert_bits_equal(y, oracle.apply(A.n, ref["rowptr"], ref["colind"], ref["val"], p), "apply")
    trp, tci, tv = oracle.transpose(A.n, ref["rowptr"], ref["colind"], ref["val"])
    yt = F.apply(pd, transpose=True)
    assert_bits_equal(yt, oracle.apply_t(A.n, trp, tci, tv, p), "apply transpose")
    assert F.status() == L.OK


def test_factor_equals_two_calls_band_160k():
    pr = W.random_band_160k(2)
    rp, ci, av = to_dev(pr.A)
    S, F = P.factor(rp, ci, av, 2)
    S2 = P.symbolic(rp, ci, 2)
    F2 = P.numeric(S2, av)
    for a, b in zip(S.pattern(), S2.pattern()):
        assert torch.equal(a, b)
    assert_bits_equal(F.values(), F2.values().cpu().numpy(), "factor values")
    # index orders against level orders: the same bits
    p, pd = vec(19, pr.A.n)
    assert_bits_equal(F.apply(pd), F2.apply(pd).cpu().numpy(), "apply")
    b = torch.from_numpy(pr.b).cuda()
    x, info = P.gmres(rp, ci, av, b, F, restart=50, rtol=1e-8)
    x2, info2 = P.gmres(rp, ci, av, b, F2, restart=50, rtol=1e-8)
    assert info.iters == info2.iters
    assert_bits_equal(x, x2.cpu().numpy(), "gmres x")
    # levels built later (depth query), then a refactorization on them
    dl, du = S.depth()
    assert (dl, du) == S2.depth()
    F.refactor(av)
    assert_bits_equal(F.values(), F2.values().cpu().numpy(), "refactor values")
    assert_bits_equal(F.apply(pd), F2.apply(pd).cpu().numpy(), "apply on level orders")


def test_factor_errors_as_the_two_calls():
    # a zero pivot in row 2 (a_22 = 0 and no update reaches it)
    A = W.dense_to_csr(np.array([[2.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 0.0]]),
                       mask=np.ones((3, 3), dtype=bool))
    rp, ci, av = to_dev(A)
    with pytest.raises(P.IlukError) as e:
        P.factor(rp, ci, av, 2)
    assert e.value.status == L.EZEROPIVOT and e.value.row == 2


def test_factor_rows_longer_than_the_numeric_slice():
    # full fill: every row of F holds 600 entries, more than the combined
    # launch's numeric rows take, so the two separate calls run instead
    A = W.random_sparse(600, 0.02, 21)
    rp, ci, av = to_dev(A)
    S, F = P.factor(rp, ci, av, 250)
    assert S.max_row > 512
    ref = oracle.factor(A, 250)
    grp, gci, _, _ = [t.cpu().numpy() for t in S.pattern()]
    assert np.array_equal(grp, ref["rowptr"]) and np.array_equal(gci, ref["colind"])
    assert_bits_equal(F.values(), ref["val"], "factor values")


def test_factor_sorted_list_walk():
    # a 3D grid too wide for the symbolic level map (row span 2 * 48^2): the
    # symbolic rows of the combined launch take the sorted-list walk
    A = W.conv_diff(48, 3, (50.0, 50.0, 50.0))
    rp, ci, av = to_dev(A)
    S, F = P.factor(rp, ci, av, 2)
    ref = oracle.factor(A, 2)
    grp, gci, glev, _ = [t.cpu().numpy() for t in S.pattern()]
    assert np.array_equal(grp, ref["rowptr"]) and np.array_equal(gci, ref["colind"])
    assert np.array_equal(glev, ref["level"])
    assert_bits_equal(F.values(), ref["val"], "factor values")
    p, pd = vec(23, A.n)
    assert_bits_equal(F.apply(pd), oracle.apply(A.n, ref["rowptr"], ref["colind"], ref["val"], p),
                      "apply")


@pytest.mark.parametrize("precond", ["none", "ilu", "iilu"])
def test_one_call_solve_bit_exact(precond):
    # solve(): factor (one launch for k = 2), optional TPIILU, then GMRES,
    # against the oracle's factorization and GMRES with the fixed-tree dots
    A = W.conv_diff(40, 2, (20.0, 20.0))
    rp, ci, av = to_dev(A)
    b, bd = vec(44, A.n)
    x, info = P.solve(rp, ci, av, bd, k=2, restart=30, rtol=1e-10, precond=precond)
    ref = oracle.factor(A, 2)
    if precond == "ilu":
        kind, Fa = oracle.PREC_ILU, (ref["rowptr"], ref["colind"], ref["val"])
    elif precond == "iilu":
        g = oracle.iiluk_build(A.n, ref["rowptr"], ref["colind"], ref["val"])
        kind, Fa = oracle.PREC_IILU, (ref["rowptr"], ref["colind"], g)
    else:
        kind, Fa = oracle.PREC_NONE, None
    st, xo, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, kind, Fa, 30, 1e-10,
                                        dotmode=oracle.DOT_TREE)
    assert st == oracle.OK and info.status == st and info.iters == it and info.cycles == cyc
    assert_bits_equal(x, xo, "solve x")
