"""The one-call solve (iluk_solve) against the oracle and against the two
calls it replaces.

iluk_solve forms GMRES's first vector v_1 = b / ||b|| before the
factorization, lets the one-launch factorization solve L x = v_1 as its rows
are factored, and starts GMRES's first preconditioner application with the
backward sweep.  None of that may change a bit: x, the iteration and cycle
counts and the reported residual must equal the oracle's factor + GMRES
(fixed-tree inner products, x0 = 0) and the library's own iluk_factor +
gmres_solve.  Covered: the one-launch path (k >= 2) on several matrix
families, the fallbacks (k <= 1; rows too long for the launch's numeric
slice, which sends the factorization to the two separate phases), several
restart cycles, every sweep schedule for the backward-only first
application, the autotuner running inside the call, the factors it returns
(usable afterwards), and the degenerate cases (b = 0, maxit = 0, a zero
pivot, a non-finite value).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0803_0048_gb300 as P
from paper_0803_0048_gb300 import _lib as L
from paper_0803_0048_gb300 import workloads as W

from gpu_helpers import assert_bits_equal, bits, to_dev, vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def oracle_solve(A, b, k, m, rtol, maxit=10000):
    ref = oracle.factor(A, k)
    out = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                       (ref["rowptr"], ref["colind"], ref["val"]), m, rtol, maxit=maxit,
                       dotmode=oracle.DOT_TREE)
    return ref, out


CASES = [
    # (name, matrix, k, restart)
    ("convdiff2d_64_k2", W.conv_diff(64, 2, (20.0, 20.0)), 2, 30),
    ("convdiff3d_12_k3", W.conv_diff(12, 3, (50.0, 50.0, 50.0)), 3, 30),
    ("band4000_k2", W.random_band(4000, 9, 200, 5), 2, 50),
    ("band3000_k2_restart4", W.random_band(3000, 9, 100, 11), 2, 4),
    ("rand1000_k3", W.random_sparse(1000, 0.006, 6), 3, 30),
    ("rand37_k2", W.random_sparse(37, 0.15, 3), 2, 10),
    ("band4000_k1", W.random_band(4000, 9, 200, 5), 1, 50),
    ("convdiff3d_12_k0", W.conv_diff(12, 3, (50.0, 50.0, 50.0)), 0, 30),
]


@pytest.mark.parametrize("name,A,k,m", CASES, ids=[c[0] for c in CASES])
def test_one_call_solve_bit_exact_vs_oracle_and_two_calls(name, A, k, m):
    rp, ci, av = to_dev(A)
    b, bd = vec(71, A.n)
    rtol = 1e-10
    ref, (st, xo, it, rel, cyc) = oracle_solve(A, b, k, m, rtol)
    assert st == 0
    x, info, (S, F) = P.solve(rp, ci, av, bd, k=k, restart=m, rtol=rtol, return_factors=True)
    assert info.status == 0 and (info.iters, info.cycles) == (it, cyc)
    assert bits([info.relres])[0] == bits([rel])[0]
    assert_bits_equal(x, xo, f"{name}: x")
    assert_bits_equal(F.values(), ref["val"], f"{name}: factors")
    # the two calls it replaces, on the schedule the call picked
    S2, F2 = P.factor(rp, ci, av, k)
    F2.set_schedule(F.schedule())
    x2, info2 = P.gmres(rp, ci, av, bd, F2, restart=m, rtol=rtol)
    assert (info2.iters, info2.cycles) == (info.iters, info.cycles)
    assert_bits_equal(x2, x.cpu().numpy(), f"{name}: factor + gmres")
    # the returned factors are left ready for other applies and solves
    p, pd = vec(72, A.n)
    assert_bits_equal(F.apply(pd), oracle.apply(A.n, ref["rowptr"], ref["colind"], ref["val"], p),
                      f"{name}: apply after the call")
    x3, _ = P.gmres(rp, ci, av, bd, F, restart=m, rtol=rtol)
    assert_bits_equal(x3, xo, f"{name}: gmres on the returned factors")


SCHEDS = [L.SCHED_FLAGS, L.SCHED_SINGLE_CTA, L.SCHED_CLUSTER, L.SCHED_WARP_GRID,
          L.SCHED_WARP_CLUSTER, L.sched_width(L.SCHED_WARP_GRID, 256),
          L.sched_width(L.SCHED_WARP_CLUSTER, 512),
          L.SCHED_SINGLE_CTA | (L.sched_width(L.SCHED_WARP_CLUSTER, 256) << 8),
          L.sched_width(L.SCHED_WARP_CLUSTER, 384) | (L.SCHED_FLAGS << 8),
          L.sched_width(L.SCHED_WARP_CLUSTER_HELP, 512),
          L.sched_width(L.SCHED_WARP_CLUSTER_HELP, 384) | (L.SCHED_WARP_CLUSTER << 8)]


@pytest.mark.parametrize("sched", SCHEDS)
def test_one_call_solve_every_schedule(sched):
    """The first application's backward-only sweep under every schedule
    (forward and backward bytes apart or together)."""
    A = W.conv_diff(40, 2, (20.0, 20.0))
    rp, ci, av = to_dev(A)
    b, bd = vec(73, A.n)
    _, (st, xo, it, rel, cyc) = oracle_solve(A, b, 2, 20, 1e-10)
    x, info = P.solve(rp, ci, av, bd, k=2, restart=20, rtol=1e-10, sched=sched)
    assert info.status == 0 and (info.iters, info.cycles) == (it, cyc)
    assert bits([info.relres])[0] == bits([rel])[0]
    assert_bits_equal(x, xo, f"schedule {sched:#x}")


def test_one_call_solve_rows_longer_than_the_numeric_slice():
    """Full fill (rows of 600 entries): the one-launch factorization hands the
    work to the two separate phases, so the first application runs both
    sweeps; same bits as the oracle."""
    A = W.random_sparse(600, 0.02, 21)
    rp, ci, av = to_dev(A)
    b, bd = vec(74, A.n)
    ref, (st, xo, it, rel, cyc) = oracle_solve(A, b, 3, 30, 1e-10)
    assert int(np.diff(ref["rowptr"]).max()) > 512
    x, info = P.solve(rp, ci, av, bd, k=3, restart=30, rtol=1e-10)
    assert info.status == st and (info.iters, info.cycles) == (it, cyc)
    assert_bits_equal(x, xo, "x")


def test_one_call_solve_degenerate_cases():
    A = W.conv_diff(20, 2, (20.0, 20.0))
    rp, ci, av = to_dev(A)
    ref = oracle.factor(A, 2)
    # b = 0: x = 0 with no iteration, and the factorization still runs
    z = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    x, info, (S, F) = P.solve(rp, ci, av, z, k=2, return_factors=True)
    assert info.status == 0 and info.iters == 0 and not torch.any(x != 0)
    assert_bits_equal(F.values(), ref["val"], "factors with b = 0")
    # maxit = 0: no iteration, GMRES reports no convergence
    b, bd = vec(75, A.n)
    x, info = P.solve(rp, ci, av, bd, k=2, maxit=0, check=False)
    assert info.status == L.ENOCONV and info.iters == 0 and not torch.any(x != 0)
    # rtol >= 1: x0 = 0 already meets it
    x, info = P.solve(rp, ci, av, bd, k=2, rtol=1.0)
    assert info.status == 0 and info.iters == 0


def test_one_call_solve_reports_factorization_failures():
    # a zero pivot at row 2 (nothing updates a_22 = 0), found whether or not
    # GMRES gets as far as its first application
    A = W.dense_to_csr(np.array([[2.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 0.0]]),
                       mask=np.ones((3, 3), dtype=bool))
    rp, ci, av = to_dev(A)
    for bv in (np.array([1.0, 2.0, 3.0]), np.zeros(3)):
        bd = torch.from_numpy(bv).cuda()
        with pytest.raises(P.IlukError) as e:
            P.solve(rp, ci, av, bd, k=2)
        assert e.value.status == L.EZEROPIVOT and e.value.row == 2
    # a non-finite value
    A = W.random_sparse(100, 0.05, 4)
    A.val[A.rowptr[30]] = np.nan
    rp, ci, av = to_dev(A)
    b, bd = vec(76, A.n)
    with pytest.raises(P.IlukError) as e:
        P.solve(rp, ci, av, bd, k=2)
    assert e.value.status == L.ENONFINITE
    # a pattern the validation rejects (columns out of order in row 0)
    A = W.random_sparse(50, 0.1, 5)
    assert A.rowptr[1] - A.rowptr[0] >= 2
    c = A.colind.copy()
    c[A.rowptr[0]], c[A.rowptr[0] + 1] = c[A.rowptr[0] + 1], c[A.rowptr[0]]
    rp, ci, av = to_dev(W.CSR(A.n, A.rowptr, c, A.val))
    b, bd = vec(77, A.n)
    with pytest.raises(P.IlukError) as e:
        P.solve(rp, ci, av, bd, k=2)
    assert e.value.status == L.EPATTERN


def _forward_depth(ref):
    """Longest chain of the forward DAG of F's lower pattern (levels from 1)."""
    rp, ci = ref["rowptr"], ref["colind"]
    n = len(rp) - 1
    depth = np.zeros(n, dtype=np.int64)
    for i in range(n):
        lo = ci[rp[i]:rp[i + 1]]
        lo = lo[lo < i]
        depth[i] = 1 + (depth[lo].max() if lo.size else 0)
    return int(depth.max())


def _levels_built(S):
    import ctypes as C
    v = L.SymView()
    L.load().iluk_sym_query(S.h, C.byref(v))
    return v.depth_lower


@pytest.mark.parametrize("name,make,k", [
    ("convdiff3d_32_k1", lambda: W.conv_diff(32, 3, (50.0, 50.0, 50.0)), 1),   # 175 rows a level
    ("convdiff3d_40_k2", lambda: W.conv_diff(40, 3, (50.0, 50.0, 50.0)), 2),   # 149 rows a level
    ("convdiff3d_24_k2", lambda: W.conv_diff(24, 3, (50.0, 50.0, 50.0)), 2),   # 54 rows a level
    ("band20000_k2", lambda: W.random_band(20000, 9, 400, 3), 2)],            # 3 rows a level
    ids=["3d32_k1", "3d40_k2", "3d24_k2", "band20000_k2"])
def test_factorization_leaves_level_orders_on_wide_dags(name, make, k):
    """A factorization made without level orders measures the forward DAG's
    depth and builds the level orders when the DAG is wide (n >= 128 depth),
    as the one-call solve then needs; the results stay the oracle's."""
    A = make()
    rp, ci, av = to_dev(A)
    b, bd = vec(78, A.n)
    ref, (st, xo, it, rel, cyc) = oracle_solve(A, b, k, 30, 1e-10)
    depth = _forward_depth(ref)
    wide = A.n >= 128 * depth
    S, F = P.factor(rp, ci, av, k)
    got = _levels_built(S)
    if wide:
        assert got == depth, (got, depth)
    else:
        assert got == -1
    assert_bits_equal(F.values(), ref["val"], f"{name}: factors")
    x, info = P.solve(rp, ci, av, bd, k=k, restart=30, rtol=1e-10)
    assert (info.iters, info.cycles) == (it, cyc)
    assert_bits_equal(x, xo, f"{name}: one-call solve")
