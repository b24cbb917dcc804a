"""Device-side error reporting: bad inputs are turned into statuses, never into
GPU faults, and every row-to-row wait is bounded.

All failures are made on the host (bad CSR arrays, a zero pivot, a NaN, a row
whose completion is withheld by the test hook); none of them faults or hangs
the GPU.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0803_0048_gb300 as P
from paper_0803_0048_gb300 import _lib as L
from paper_0803_0048_gb300 import workloads as W

from gpu_helpers import assert_bits_equal, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def dev_pattern(rp, ci):
    return (torch.tensor(rp, dtype=torch.int64, device="cuda"),
            torch.tensor(ci, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("rp,ci,row", [
    ([0, 2, 3], [1, 0, 1], 0),        # unsorted
    ([0, 2, 3], [0, 0, 1], 0),        # duplicate
    ([0, 1, 3], [0, 0, 2], 1),        # out of range
    ([0, 2, 1, 3], [0, 1, 1], 1),     # decreasing rowptr
    ([0, 2, 3], [0, 1], 0),           # rowptr[n] != nnz
])
def test_bad_patterns_rejected(rp, ci, row):
    r, c = dev_pattern(rp, ci)
    st, bad = P.validate(r, c)
    assert st == L.EPATTERN and bad == row
    with pytest.raises(P.IlukError) as e:
        P.symbolic(r, c, 1)
    assert e.value.status == L.EPATTERN


def test_missing_diagonal_and_fill_diagonal():
    A = W.dense_to_csr(np.array([[1.0, 1.0, 0.0], [1.0, 0.0, 1.0], [0.0, 1.0, 1.0]]))
    rp, ci, av = to_dev(A)
    with pytest.raises(P.IlukError) as e:
        P.symbolic(rp, ci, 0)
    assert e.value.status == L.ENODIAG and e.value.row == 1
    S = P.symbolic(rp, ci, 1)  # (1,1) enters as a level-1 fill through h = 0
    _, _, lev, dg = S.pattern()
    assert lev[dg[1]].item() == 1


def test_zero_pivot_reports_first_row():
    n = 300
    A = W.random_sparse(n, 0.02, 3)
    D = W.csr_to_dense(A)
    D[40, 40] = 0.0
    D[200, 200] = 0.0
    mask = W.csr_to_dense(A) != 0
    A2 = W.dense_to_csr(D, mask)
    st, bad, frp, fci, _ = oracle.symbolic(n, A2.rowptr, A2.colind, 1)
    st, bad, _ = oracle.numeric(n, A2.rowptr, A2.colind, A2.val, frp, fci)
    rp, ci, av = to_dev(A2)
    S = P.symbolic(rp, ci, 1)
    with pytest.raises(P.IlukError) as e:
        P.numeric(S, av)
    assert e.value.status == L.EZEROPIVOT == st
    assert e.value.row == bad


def test_nonfinite_value():
    A = W.random_sparse(100, 0.05, 4)
    A.val[A.rowptr[30]] = np.nan
    rp, ci, av = to_dev(A)
    S = P.symbolic(rp, ci, 2)
    with pytest.raises(P.IlukError) as e:
        P.numeric(S, av)
    assert e.value.status == L.ENONFINITE and e.value.row == 30


def test_bounded_wait_times_out_and_gpu_stays_usable():
    A = W.conv_diff(16, 2, (1.0, 1.0))
    rp, ci, av = to_dev(A)
    S = P.symbolic(rp, ci, 1)
    old = P.set_wait_limit(50_000_000)  # 50 ms
    P.debug_hold_row(100)
    try:
        with pytest.raises(P.IlukError) as e:
            P.numeric(S, av)
        assert e.value.status == L.ETIMEOUT
        assert e.value.row > 100
    finally:
        P.debug_hold_row(-1)
        P.set_wait_limit(old)
    F = P.numeric(S, av)  # the context is still healthy
    ref = oracle.factor(A, 1)
    assert np.array_equal(F.values().cpu().numpy(), ref["val"])


def test_empty_and_single_row():
    rp, ci = dev_pattern([0], [])
    S = P.symbolic(rp, ci, 2)
    assert S.n == 0 and S.nnz == 0
    rp, ci = dev_pattern([0, 1], [0])
    S = P.symbolic(rp, ci, 2)
    F = P.numeric(S, torch.tensor([4.0], dtype=torch.float64, device="cuda"))
    y = F.apply(torch.tensor([2.0], dtype=torch.float64, device="cuda"))
    assert y.item() == 0.5


def test_gmres_reports_nonconvergence():
    A = W.conv_diff(20, 2, (20.0, 20.0))
    rp, ci, av = to_dev(A)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    x, info = P.gmres(rp, ci, av, b, None, restart=5, rtol=1e-12, maxit=12, check=False)
    assert info.status == L.ENOCONV and info.iters == 12


def test_tuned_schedule_kept_by_the_pattern():
    """The first GMRES on a factorization times the sweep schedules; a later
    factorization of the same pattern (new values) starts from that pick and
    times nothing, and its results are those of the oracle either way."""
    A = W.random_band(3000, 9, 100, 17)
    rp, ci, av = to_dev(A)
    S = P.symbolic(rp, ci, 2)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    F1 = P.numeric(S, av)
    c0 = P.launch_count()
    x1, i1 = P.gmres(rp, ci, av, b, F1, restart=20, rtol=1e-10)
    tuned_launches = P.launch_count() - c0
    s1 = F1.schedule()
    assert s1 != L.SCHED_AUTO
    av2 = av * 1.5  # other values, same pattern
    F2 = P.numeric(S, av2)
    assert F2.schedule() == L.SCHED_AUTO  # nothing fixed on the new factors yet
    c0 = P.launch_count()
    x2, i2 = P.gmres(rp, ci, av2, b, F2, restart=20, rtol=1e-10)
    launches = P.launch_count() - c0
    assert F2.schedule() == s1
    # the timing runs (13 kinds/widths, 3 runs of 2 sweeps each) are gone
    assert tuned_launches - launches >= 40, (tuned_launches, launches)
    A2 = W.CSR(A.n, A.rowptr, A.colind, A.val * 1.5)
    ref = oracle.factor(A2, 2)
    st, xo, it, rel, cyc = oracle.gmres(A2.n, A2.rowptr, A2.colind, A2.val, np.ones(A.n),
                                        oracle.PREC_ILU, (ref["rowptr"], ref["colind"], ref["val"]),
                                        20, 1e-10, dotmode=oracle.DOT_TREE)
    assert i2.iters == it
    assert_bits_equal(x2, xo, "second factorization's solve")
    # the transposed sweeps (A^T lambda = g) are timed on their own, once
    c0 = P.launch_count()
    P.gmres(rp, ci, av2, b, F2, restart=20, rtol=1e-10, transpose=True)
    tuned_t = P.launch_count() - c0
    F3 = P.numeric(S, av)
    P.gmres(rp, ci, av, b, F3, restart=20, rtol=1e-10)  # schedule from the pattern
    c0 = P.launch_count()
    lam, it3 = P.gmres(rp, ci, av, b, F3, restart=20, rtol=1e-10, transpose=True)
    assert tuned_t - (P.launch_count() - c0) >= 40
    r1 = oracle.factor(A, 2)
    x1o = oracle.gmres(A.n, A.rowptr, A.colind, A.val, np.ones(A.n), oracle.PREC_ILU,
                       (r1["rowptr"], r1["colind"], r1["val"]), 20, 1e-10,
                       dotmode=oracle.DOT_TREE)[1]
    st, lo, _, itt, _ = oracle.adjoint(A.n, A.rowptr, A.colind, A.val, r1["rowptr"],
                                       r1["colind"], r1["val"], x1o, np.ones(A.n), 20, 1e-10,
                                       dotmode=oracle.DOT_TREE)
    assert st == oracle.OK and it3.iters == itt
    assert_bits_equal(lam, lo, "transposed solve with the pattern's schedule")


def test_schedule_values_checked():
    A = W.conv_diff(12, 2, (20.0, 20.0))
    rp, ci, av = to_dev(A)
    F = P.numeric(P.symbolic(rp, ci, 1), av)
    good = [L.SCHED_AUTO, L.SCHED_FLAGS, L.sched_width(L.SCHED_WARP_CLUSTER, 256),
            L.sched_width(L.SCHED_WARP_GRID, 1024),
            L.SCHED_CLUSTER | (L.sched_width(L.SCHED_WARP_CLUSTER, 768) << 8),
            L.SCHED_WARP_CLUSTER_HELP, L.sched_width(L.SCHED_WARP_CLUSTER_HELP, 384)]
    for s in good:
        F.set_schedule(s)
        assert F.schedule() == s
    bad = [7, 0x0F, L.sched_width(L.SCHED_FLAGS, 512),  # width on a lockstep kind
           L.SCHED_WARP_GRID | (1 << 4), L.SCHED_WARP_GRID | (9 << 4),  # 128 / 1152 threads
           L.SCHED_WARP_CLUSTER_HELP | (9 << 4),
           L.SCHED_WARP_GRID | (7 << 8), -1, 1 << 16]
    for s in bad:
        with pytest.raises(P.IlukError):
            F.set_schedule(s)
