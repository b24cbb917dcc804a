"""GPU tests of the two additions beyond the single solve:

* a7 batched persistent solve: every item of a batch (one shared pattern with
  several value sets, plus grids of other sizes) must be bit-identical to the
  single-instance path, including after capture into a CUDA graph and replay
  with new values;
* a8 differentiable solve: the hand-written adjoint must match the oracle's
  adjoint bit for bit (fixed-tree inner products), and central finite
  differences of the loss within 1e-5 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0803_0048_gb300 as P
from paper_0803_0048_gb300 import _lib as L
from paper_0803_0048_gb300 import workloads as W

from gpu_helpers import assert_bits_equal, bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def fd_instance(N, seed, d=3):
    Pt = W.fd_pattern(N, d)
    th = W.log_uniform(W.stream_key(seed, "bt"), np.arange(Pt.n), 0.1, 10.0)
    beta = W.uniform(W.stream_key(seed, "bb"), np.arange(d), 0.0, 30.0)
    vals = W.fd_values(Pt, torch.from_numpy(th), [float(v) for v in beta]).numpy()
    b = W.uniform(W.stream_key(seed, "rhs"), np.arange(Pt.n), -1.0, 1.0)
    return Pt, vals, b


def build_batch(k=1):
    items, host = [], []
    shared = W.fd_pattern(9, 3)
    rp = torch.from_numpy(shared.rowptr).cuda()
    ci = torch.from_numpy(shared.colind).cuda()
    S_shared = P.symbolic(rp, ci, k)
    for s in range(5):
        _, vals, b = fd_instance(9, 100 + s)
        items.append((S_shared, torch.from_numpy(vals).cuda(), torch.from_numpy(b).cuda(),
                      torch.empty(shared.n, dtype=torch.float64, device="cuda")))
        host.append((rp, ci))
    for N in (6, 11, 13):
        Pt, vals, b = fd_instance(N, 200 + N)
        r = torch.from_numpy(Pt.rowptr).cuda()
        c = torch.from_numpy(Pt.colind).cuda()
        S = P.symbolic(r, c, k)
        items.append((S, torch.from_numpy(vals).cuda(), torch.from_numpy(b).cuda(),
                      torch.empty(Pt.n, dtype=torch.float64, device="cuda")))
        host.append((r, c))
    return items, host


def single_solve(S, rp, ci, vals, b, restart, rtol):
    F = P.numeric(S, vals)
    x, info = P.gmres(rp, ci, vals, b, F, restart=restart, rtol=rtol, check=False)
    return x, info


def test_batched_solve_bit_exact_vs_single():
    items, host = build_batch()
    B = P.BatchSolve(items, restart=30, rtol=1e-8)
    B.solve()
    res = B.results()
    assert B.width() in (256, 512, 1024)
    for (S, vals, b, x), (rp, ci), r in zip(items, host, res):
        xs, info = single_solve(S, rp, ci, vals, b, 30, 1e-8)
        assert r.status == info.status == 0
        assert r.iters == info.iters and r.cycles == info.cycles
        assert bits([r.relres])[0] == bits([info.relres])[0]
        assert_bits_equal(x, xs, "batched x")


def test_batched_solve_graph_capture_and_replay():
    items, host = build_batch()
    B = P.BatchSolve(items, restart=30, rtol=1e-8)
    B.solve()  # first call outside the capture runs the autotuner
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.solve()
    # new values in the same buffers, then replay
    for i, (S, vals, b, x) in enumerate(items):
        vals.mul_(1.0 + 0.125 * (i % 3))
        b.mul_(-0.5)
        x.zero_()
    g.replay()
    torch.cuda.synchronize()
    res = B.results()
    for (S, vals, b, x), (rp, ci), r in zip(items, host, res):
        xs, info = single_solve(S, rp, ci, vals, b, 30, 1e-8)
        assert r.status == 0 and r.iters == info.iters
        assert_bits_equal(x, xs, "replayed x")


@pytest.mark.parametrize("sched", [None, (256, False), (256, True), (512, False), (512, True),
                                   (1024, False), (1024, True)],
                         ids=["auto", "256-level", "256-spin", "512-level", "512-spin",
                              "1024-level", "1024-spin"])
def test_batched_solve_reports_factorization_errors_per_item(sched):
    """A zero pivot and a non-finite value of A, each in its own item, are
    reported for that item with the row (the smallest offending one), under
    every schedule (rows factored by half-warp pairs and by whole warps); the
    other items solve as usual."""
    items, host = build_batch()
    items[2][1].zero_()  # all-zero matrix: zero pivot at row 0
    S, vals, b, x = items[6]  # the 11^3 grid
    bad_row = 700
    rp = host[6][0]
    vals[int(rp[bad_row].item()) + 1] = float("nan")
    B = P.BatchSolve(items, restart=30, rtol=1e-8)
    if sched is not None:
        B.set_schedule(*sched)
    B.solve()
    res = B.results()
    assert res[2].status == L.EZEROPIVOT and res[2].row == 0
    assert res[6].status == L.ENONFINITE and res[6].row == bad_row
    assert all(r.status == 0 for i, r in enumerate(res) if i not in (2, 6))


def adjoint_setup(N=12, k=2):
    Pt = W.fd_pattern(N, 2)
    n = Pt.n
    theta0 = W.log_uniform(W.stream_key(5, "adj"), np.arange(n), 0.1, 10.0)
    beta = (20.0, 20.0)
    b = W.uniform(W.stream_key(5, "adjb"), np.arange(n), -1.0, 1.0)
    xt = W.uniform(W.stream_key(5, "adjx"), np.arange(n), -1.0, 1.0)
    rp = torch.from_numpy(Pt.rowptr).cuda()
    ci = torch.from_numpy(Pt.colind).cuda()
    return Pt, theta0, beta, b, xt, rp, ci


def test_adjoint_bit_exact_vs_oracle():
    Pt, theta0, beta, b, xt, rp, ci = adjoint_setup()
    solver = P.IlukSolver(rp, ci, k=2, restart=30, rtol=1e-12)
    th = torch.from_numpy(theta0).cuda().requires_grad_(True)
    bd = torch.from_numpy(b).cuda().requires_grad_(True)
    vals = W.fd_values(Pt, th, beta)
    x = solver.solve(vals, bd)
    loss = ((x - torch.from_numpy(xt).cuda()) ** 2).sum()
    loss.backward()
    # oracle adjoint on the same values
    v = vals.detach().cpu().numpy()
    A = W.CSR(Pt.n, Pt.rowptr, Pt.colind, v)
    F = oracle.factor(A, 2)
    st, xo, *_ = oracle.gmres(A.n, A.rowptr, A.colind, v, b, oracle.PREC_ILU,
                              (F["rowptr"], F["colind"], F["val"]), 30, 1e-12,
                              dotmode=oracle.DOT_TREE)
    assert_bits_equal(x.detach(), xo, "forward x")
    gx = 2.0 * (xo - xt)
    st, lam, gA, it, rel = oracle.adjoint(A.n, A.rowptr, A.colind, v, F["rowptr"], F["colind"],
                                          F["val"], xo, gx, 30, 1e-12, dotmode=oracle.DOT_TREE)
    assert st == 0
    assert_bits_equal(bd.grad, lam, "dL/db")
    # dL/dtheta from the oracle's dL/dA through the same torch assembly
    th2 = torch.from_numpy(theta0).requires_grad_(True)
    vals2 = W.fd_values(Pt, th2, beta)
    (gth,) = torch.autograd.grad(vals2, th2, grad_outputs=torch.from_numpy(gA))
    np.testing.assert_allclose(th.grad.cpu().numpy(), gth.numpy(), rtol=1e-10, atol=1e-14)
    # and within 1e-10 of the sequential-dot oracle
    st, lam_s, *_ = oracle.adjoint(A.n, A.rowptr, A.colind, v, F["rowptr"], F["colind"],
                                   F["val"], xo, gx, 30, 1e-12, dotmode=oracle.DOT_SEQ)
    assert np.linalg.norm(bd.grad.cpu().numpy() - lam_s) <= 1e-10 * np.linalg.norm(lam_s)


def test_adjoint_matches_central_finite_differences():
    Pt, theta0, beta, b, xt, rp, ci = adjoint_setup(N=10)
    solver = P.IlukSolver(rp, ci, k=2, restart=30, rtol=1e-13)
    xtd = torch.from_numpy(xt).cuda()

    def loss_of(theta, bb, grad=False):
        th = torch.from_numpy(theta).cuda().requires_grad_(grad)
        bd = torch.from_numpy(bb).cuda().requires_grad_(grad)
        x = solver.solve(W.fd_values(Pt, th, beta), bd)
        L = ((x - xtd) ** 2).sum()
        if grad:
            L.backward()
            return float(L.detach()), th.grad.cpu().numpy(), bd.grad.cpu().numpy()
        return float(L.detach())

    L0, gth, gb = loss_of(theta0, b, grad=True)
    for c in (0, 11, 37, 55, 99):
        h = 1e-6 * theta0[c]
        tp, tm = theta0.copy(), theta0.copy()
        tp[c] += h
        tm[c] -= h
        fd = (loss_of(tp, b) - loss_of(tm, b)) / (2 * h)
        assert abs(fd - gth[c]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gth).max())
    for c in (3, 48, 90):
        h = 1e-6
        bp, bm = b.copy(), b.copy()
        bp[c] += h
        bm[c] -= h
        fd = (loss_of(theta0, bp) - loss_of(theta0, bm)) / (2 * h)
        assert abs(fd - gb[c]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gb).max())


@pytest.mark.parametrize("width", [256, 512, 1024])
@pytest.mark.parametrize("spin", [False, True])
def test_batched_every_schedule_bit_exact_vs_single(width, spin):
    items, host = build_batch()
    B = P.BatchSolve(items, restart=30, rtol=1e-8)
    B.set_schedule(width, spin)
    B.solve()
    res = B.results()
    assert B.width() == width and B.spin() == spin
    for (S, vals, b, x), (rp, ci), r in zip(items, host, res):
        xs, info = single_solve(S, rp, ci, vals, b, 30, 1e-8)
        assert r.status == info.status == 0 and r.iters == info.iters
        assert_bits_equal(x, xs, "batched x")
