"""GPU parity: the CUDA library against the sequential oracle, element by
element on the same seeded inputs.

Integer results (pattern, levels) must be bit-exact; so must every floating
point result, because both sides perform the same IEEE operations in the same
per-entry order (the paper's bit-compatibility property, Sec. 1).  GMRES is
bit-exact against the oracle's fixed-tree inner product and within 1e-10 of
its sequential inner product.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0803_0048_gb300 as P
from paper_0803_0048_gb300 import _lib as L
from paper_0803_0048_gb300 import workloads as W

from gpu_helpers import assert_bits_equal, bits, small_cases, to_dev, vec

pytestmark = pytest.mark.gpu

CASES = small_cases()
IDS = [c[0] for c in CASES]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def factor_both(A, k):
    rp, ci, av = to_dev(A)
    S = P.symbolic(rp, ci, k)
    F = P.numeric(S, av)
    ref = oracle.factor(A, k)
    return S, F, ref, (rp, ci, av)


@pytest.mark.parametrize("name,A,k", CASES, ids=IDS)
def test_symbolic_matches_oracle(name, A, k):
    rp, ci, _ = to_dev(A)
    S = P.symbolic(rp, ci, k)
    st, bad, frp, fci, flev = oracle.symbolic(A.n, A.rowptr, A.colind, k)
    assert st == oracle.OK
    grp, gci, glev, gdg = [t.cpu().numpy() for t in S.pattern()]
    assert np.array_equal(grp, frp)
    assert np.array_equal(gci, fci)
    assert np.array_equal(glev, flev)
    for i in range(A.n):
        assert gci[gdg[i]] == i
    assert S.max_row == int(np.diff(frp).max(initial=0))


@pytest.mark.parametrize("name,A,k", CASES, ids=IDS)
def test_numeric_bit_exact(name, A, k):
    S, F, ref, _ = factor_both(A, k)
    assert_bits_equal(F.values(), ref["val"], "factor values")


SCHEDS = [L.SCHED_FLAGS, L.SCHED_SINGLE_CTA, L.SCHED_CLUSTER, L.SCHED_WARP_GRID,
          L.SCHED_WARP_CLUSTER, L.sched_width(L.SCHED_WARP_GRID, 256),
          L.sched_width(L.SCHED_WARP_CLUSTER, 384),
          # forward and backward on different schedules
          L.SCHED_SINGLE_CTA | (L.sched_width(L.SCHED_WARP_CLUSTER, 256) << 8),
          # with the prefix-helper cluster
          L.SCHED_WARP_CLUSTER_HELP, L.sched_width(L.SCHED_WARP_CLUSTER_HELP, 384),
          L.sched_width(L.SCHED_WARP_CLUSTER_HELP, 512) | (L.SCHED_WARP_GRID << 8),
          # invalid kind and width: fall back to the warp grid
          0x9F]


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("name,A,k", CASES, ids=IDS)
def test_apply_bit_exact(name, A, k, sched):
    S, F, ref, _ = factor_both(A, k)
    p, pd = vec(17, A.n)
    y = F.apply(pd, sched=sched)
    want = oracle.apply(A.n, ref["rowptr"], ref["colind"], ref["val"], p)
    assert_bits_equal(y, want, "apply")
    trp, tci, tv = oracle.transpose(A.n, ref["rowptr"], ref["colind"], ref["val"])
    yt = F.apply(pd, transpose=True, sched=sched)
    want_t = oracle.apply_t(A.n, trp, tci, tv, p)
    assert_bits_equal(yt, want_t, "apply transpose")
    assert F.status() == L.OK


@pytest.mark.parametrize("name,A,k", CASES, ids=IDS)
def test_tpiilu_bit_exact(name, A, k):
    S, F, ref, _ = factor_both(A, k)
    M = P.iiluk_build(F)
    g = oracle.iiluk_build(A.n, ref["rowptr"], ref["colind"], ref["val"])
    assert_bits_equal(M.values(), g, "TPIILU g")
    p, pd = vec(23, A.n)
    y = M.apply(pd)
    assert_bits_equal(y, oracle.iiluk_apply(A.n, ref["rowptr"], ref["colind"], g, p), "iilu apply")


def test_spmv_and_dot_bit_exact():
    A = W.random_band(5000, 9, 300, 3)
    rp, ci, av = to_dev(A)
    x, xd = vec(5, A.n)
    assert_bits_equal(P.spmv(rp, ci, av, xd), oracle.spmv(A.n, A.rowptr, A.colind, A.val, x))
    # the GPU reduction takes rows of 4096 in chunks of 48 rows (196,608
    # elements): sizes below, at and across chunk boundaries, ragged tails
    for n in (0, 1, 4095, 4096, 4097, 100003, 196608, 196609, 393216 + 4095, 600011):
        a, ad = vec(6, n)
        b, bd = vec(7, n)
        got = P.dot(ad, bd).item()
        assert bits([got])[0] == bits([oracle.dot(a, b, oracle.DOT_TREE)])[0]


def test_gmres_bit_exact_multi_chunk():
    # n spans three chunks of the reduction kernels (w <- w - h v fused with
    # the next inner product, and ||w|| on the last step): a fixed budget of
    # iterations without a preconditioner, compared bit for bit
    A = W.random_band(420011, 5, 40, 9)
    rp, ci, av = to_dev(A)
    b, bd = vec(33, A.n)
    x, info = P.gmres(rp, ci, av, bd, None, restart=8, rtol=1e-14, maxit=20, check=False)
    st, xo, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_NONE,
                                        None, 8, 1e-14, maxit=20, dotmode=oracle.DOT_TREE)
    assert info.status == st and info.iters == it == 20 and info.cycles == cyc
    assert bits([info.relres])[0] == bits([rel])[0]
    assert_bits_equal(x, xo, "gmres x")


GMRES_CASES = [
    ("convdiff2d_64_k2", W.conv_diff(64, 2, (20.0, 20.0)), 2, 30),
    ("convdiff3d_12_k1", W.conv_diff(12, 3, (50.0, 50.0, 50.0)), 1, 50),
    ("band4000_k1", W.random_band(4000, 9, 200, 5), 1, 50),
]


@pytest.mark.parametrize("prec", ["none", "ilu", "iilu"])
@pytest.mark.parametrize("name,A,k,m", GMRES_CASES, ids=[c[0] for c in GMRES_CASES])
def test_gmres_bit_exact_vs_tree_oracle(name, A, k, m, prec):
    S, F, ref, (rp, ci, av) = factor_both(A, k)
    b, bd = vec(31, A.n)
    if prec == "ilu":
        pr, kind, Fa = F, oracle.PREC_ILU, (ref["rowptr"], ref["colind"], ref["val"])
    elif prec == "iilu":
        pr = P.iiluk_build(F)
        g = oracle.iiluk_build(A.n, ref["rowptr"], ref["colind"], ref["val"])
        kind, Fa = oracle.PREC_IILU, (ref["rowptr"], ref["colind"], g)
    else:
        pr, kind, Fa = None, oracle.PREC_NONE, None
    maxit = 400
    x, info = P.gmres(rp, ci, av, bd, pr, restart=m, rtol=1e-8, maxit=maxit, check=False)
    st, xo, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, kind, Fa, m, 1e-8,
                                        maxit=maxit, dotmode=oracle.DOT_TREE)
    assert info.status == st and info.iters == it and info.cycles == cyc
    assert bits([info.relres])[0] == bits([rel])[0]
    assert_bits_equal(x, xo, "gmres x")
    st2, xs, it2, *_ = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, kind, Fa, m, 1e-8,
                                    maxit=maxit, dotmode=oracle.DOT_SEQ)
    if st == oracle.OK and st2 == oracle.OK:
        xg = x.cpu().numpy()
        rel_diff = np.linalg.norm(xg - xs) / np.linalg.norm(xs)
        if it2 == it:
            assert rel_diff <= 1e-10
        else:  # different stopping step: both meet the 1e-8 residual
            assert rel_diff <= 1e-5


def test_gmres_transpose_and_adjoint_bit_exact():
    A = W.conv_diff(20, 2, (20.0, 20.0))
    S, F, ref, (rp, ci, av) = factor_both(A, 2)
    b, bd = vec(41, A.n)
    x, info = P.gmres(rp, ci, av, bd, F, restart=30, rtol=1e-10)
    g, gd = vec(42, A.n)
    lam, info_t = P.gmres(rp, ci, av, gd, F, restart=30, rtol=1e-10, transpose=True)
    gA = P.adjoint_scatter(rp, ci, lam, x)
    st, xo, *_ = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                              (ref["rowptr"], ref["colind"], ref["val"]), 30, 1e-10,
                              dotmode=oracle.DOT_TREE)
    assert_bits_equal(x, xo, "forward x")
    st, lo, gAo, it, rel = oracle.adjoint(A.n, A.rowptr, A.colind, A.val, ref["rowptr"],
                                          ref["colind"], ref["val"], xo, g, 30, 1e-10,
                                          dotmode=oracle.DOT_TREE)
    assert st == oracle.OK and info_t.iters == it
    assert_bits_equal(lam, lo, "lambda")
    assert_bits_equal(gA, gAo, "dL/dA")


def test_batched_numeric_matches_single():
    Pt = W.fd_pattern(10, 3)
    rows = []
    for s in range(6):
        th = W.log_uniform(W.stream_key(s, "th"), np.arange(Pt.n), 0.1, 10.0)
        beta = W.uniform(W.stream_key(s, "be"), np.arange(3), 0.0, 30.0)
        rows.append(W.fd_values(Pt, torch.from_numpy(th), [float(v) for v in beta]).numpy())
    vals = np.stack(rows)
    rp = torch.from_numpy(Pt.rowptr).cuda()
    ci = torch.from_numpy(Pt.colind).cuda()
    S = P.symbolic(rp, ci, 1)
    Fb, sts = P.numeric_batched(S, torch.from_numpy(vals).cuda())
    assert sts == [0] * 6
    for s in range(6):
        F = P.numeric(S, torch.from_numpy(vals[s]).cuda())
        assert_bits_equal(Fb[s], F.values(), f"set {s}")
        ref = oracle.factor(W.CSR(Pt.n, Pt.rowptr, Pt.colind, vals[s]), 1)
        assert_bits_equal(Fb[s], ref["val"], f"set {s} vs oracle")


@pytest.mark.parametrize("prec", ["none", "ilu", "iilu"])
@pytest.mark.parametrize("name,A,k,m", GMRES_CASES, ids=[c[0] for c in GMRES_CASES])
def test_bicgstab_bit_exact_vs_tree_oracle(name, A, k, m, prec):
    S, F, ref, (rp, ci, av) = factor_both(A, k)
    b, bd = vec(51, A.n)
    if prec == "ilu":
        pr, kind, Fa = F, oracle.PREC_ILU, (ref["rowptr"], ref["colind"], ref["val"])
    elif prec == "iilu":
        pr = P.iiluk_build(F)
        g = oracle.iiluk_build(A.n, ref["rowptr"], ref["colind"], ref["val"])
        kind, Fa = oracle.PREC_IILU, (ref["rowptr"], ref["colind"], g)
    else:
        pr, kind, Fa = None, oracle.PREC_NONE, None
    maxit = 800
    x, info = P.bicgstab(rp, ci, av, bd, pr, rtol=1e-8, maxit=maxit, check=False)
    st, xo, it, rel, half = oracle.bicgstab(A.n, A.rowptr, A.colind, A.val, b, kind, Fa, 1e-8,
                                            maxit, oracle.DOT_TREE)
    assert info.status == st and info.iters == it
    assert bits([info.relres])[0] == bits([rel])[0]
    assert_bits_equal(x, xo, "bicgstab x")
    st2, xs, it2, rel2, _ = oracle.bicgstab(A.n, A.rowptr, A.colind, A.val, b, kind, Fa, 1e-8,
                                            maxit, oracle.DOT_SEQ)
    if st == oracle.OK and st2 == oracle.OK:
        rel_diff = np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs)
        if it2 == it:
            assert rel_diff <= 1e-10
        else:  # different stopping step: both meet the 1e-8 residual
            assert rel_diff <= 1e-5


def test_bicgstab_zero_rhs_and_breakdown_statuses():
    A = W.conv_diff(10, 2, (20.0, 20.0))
    rp, ci, av = to_dev(A)
    z = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    x, info = P.bicgstab(rp, ci, av, z)
    assert info.status == L.OK and info.iters == 0 and not torch.any(x)
    b, bd = vec(52, A.n)
    x, info = P.bicgstab(rp, ci, av, bd, rtol=1e-14, maxit=3, check=False)
    assert info.status == L.ENOCONV and info.iters == 3


@pytest.mark.parametrize("solver", ["gmres", "bicgstab"])
@pytest.mark.parametrize("budget,expect", [(400, "iilu"), (2, "ilu")])
def test_tpilu_policy_bit_exact(solver, budget, expect):
    Pb = W.poisson27_problem(14, k=1)
    A = Pb.A
    S, F, ref, (rp, ci, av) = factor_both(A, 1)
    b, bd = vec(61, A.n)
    x, info, used = P.tpilu_solve(rp, ci, av, bd, F, solver=solver, restart=30, rtol=1e-8,
                                  iilu_maxit=budget, maxit=400)
    g = oracle.iiluk_build(A.n, ref["rowptr"], ref["colind"], ref["val"])
    st, xo, it, rel, used_o = oracle.tpilu(A.n, A.rowptr, A.colind, A.val, b,
                                           (ref["rowptr"], ref["colind"], ref["val"]), g, solver,
                                           30, 1e-8, budget, 400, oracle.DOT_TREE)
    assert used == used_o == expect
    assert info.status == st and info.iters == it
    assert bits([info.relres])[0] == bits([rel])[0]
    assert_bits_equal(x, xo, "tpilu x")


@pytest.mark.parametrize("name,A", [("rand301", W.random_sparse(301, 0.02, 5)),
                                    ("convdiff3d_9", W.conv_diff(9, 3, (50.0, 50.0, 50.0))),
                                    ("band3000", W.random_band(3000, 9, 100, 11))],
                         ids=["rand301", "convdiff3d_9", "band3000"])
def test_transpose_matches_oracle(name, A):
    rp, ci, av = to_dev(A)
    trp, tci, tv = P.transpose(rp, ci, av)
    orp, oci, ov = oracle.transpose(A.n, A.rowptr, A.colind, A.val)
    assert np.array_equal(trp.cpu().numpy(), orp) and np.array_equal(tci.cpu().numpy(), oci)
    assert_bits_equal(tv, ov, "transposed values")


@pytest.mark.parametrize("k", [1, 2])
def test_solve_host_matches_oracle(k):
    """The host-buffer call (iluk_solve_host): host arrays in, x out on the
    host, bit-identical to the oracle's factor + GMRES with fixed-tree dots."""
    A = W.conv_diff(20, 2, (20.0, 20.0))
    b = W.uniform(W.stream_key(41, "host"), np.arange(A.n), -1.0, 1.0)
    t = [torch.from_numpy(a).pin_memory() for a in (A.rowptr, A.colind, A.val, b)]
    x, info = P.solve_host(*t, k, restart=30, rtol=1e-10)
    assert x.device.type == "cpu" and info.status == 0
    ref = oracle.factor(A, k)
    st, xo, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                                        (ref["rowptr"], ref["colind"], ref["val"]), 30, 1e-10,
                                        dotmode=oracle.DOT_TREE)
    assert (info.iters, info.cycles) == (it, cyc) and bits([info.relres])[0] == bits([rel])[0]
    assert_bits_equal(x, xo, "host-buffer solve")
    # pageable host memory works too
    x2, _ = P.solve_host(*[torch.from_numpy(a) for a in (A.rowptr, A.colind, A.val, b)], k,
                         restart=30, rtol=1e-10)
    assert_bits_equal(x2, xo, "host-buffer solve, pageable")


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("k", [0, 1])
def test_symbolic_variants_for_k_le_1_match_oracle(variant, k):
    """The k <= 1 walks (last row first; the general walk with waits) give
    the oracle's pattern and levels, through iluk_symbolic and iluk_factor."""
    cases = [W.random_sparse(301, 0.02, 5), W.conv_diff(9, 3, (50.0, 50.0, 50.0)),
             W.random_band(3000, 9, 100, 11)]
    prev = P.set_symbolic_variant(variant)
    try:
        for A in cases:
            rp, ci, av = to_dev(A)
            ref = oracle.factor(A, k)
            S = P.symbolic(rp, ci, k)
            S2, F2 = P.factor(rp, ci, av, k)
            for SS in (S, S2):
                grp, gci, glev, _ = [t.cpu().numpy() for t in SS.pattern()]
                assert np.array_equal(grp, ref["rowptr"]) and np.array_equal(gci, ref["colind"])
                assert np.array_equal(glev, ref["level"])
            assert_bits_equal(F2.values(), ref["val"], "factors")
    finally:
        P.set_symbolic_variant(prev)


@pytest.mark.parametrize("n,dens,k", [(1000, 0.01, 2), (1000, 0.01, 4), (2000, 0.004, 3),
                                      (2000, 0.004, 5)])
def test_long_rows_bit_exact(n, dens, k):
    """Random matrices that fill in to rows of hundreds to ~1,500 entries
    (the shapes of the paper's symbolic/numeric experiment): pattern, levels,
    factors and one application against the oracle, through the two phases
    and the one-call factorization."""
    A = W.random_sparse(n, dens, 77)
    rp, ci, av = to_dev(A)
    ref = oracle.factor(A, k)
    assert int(np.diff(ref["rowptr"]).max()) > 400
    S = P.symbolic(rp, ci, k)
    F = P.numeric(S, av)
    S2, F2 = P.factor(rp, ci, av, k)
    for SS, FF in ((S, F), (S2, F2)):
        grp, gci, glev, _ = [t.cpu().numpy() for t in SS.pattern()]
        assert np.array_equal(grp, ref["rowptr"]) and np.array_equal(gci, ref["colind"])
        assert np.array_equal(glev, ref["level"])
        assert_bits_equal(FF.values(), ref["val"], "factors")
    p, pd = vec(13, n)
    assert_bits_equal(F.apply(pd), oracle.apply(n, ref["rowptr"], ref["colind"], ref["val"], p),
                      "apply")
