"""GMRES(m) with the Krylov bases kept or recomputed (gmres_solve_ex).

* "recompute" keeps only V and applies the preconditioner again at the end
  of each restart cycle: x, iterations, cycles and residual must be
  bit-identical to "store" (which keeps Z = M^-1 V), and both equal the
  oracle's x += Z y form with the fixed-tree inner products, for the ILU(k)
  sweeps, TPIILU, no preconditioner and the transposed solve.
* "minv_vy" ends a cycle with x += M^-1 (V y), the textbook form of right
  preconditioning; it must equal the oracle's UPDATE_MVY mode bit for bit.
* The differentiable solve with basis="recompute" gives x and the gradients
  with respect to A's entries and b bit-identical to basis="store".
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0803_0048_gb300 as P
from paper_0803_0048_gb300 import workloads as W

from gpu_helpers import assert_bits_equal, bits, to_dev, vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


CASES = [("convdiff2d_20_k1", lambda: W.conv_diff(20, 2, (20.0, 20.0)), 1, 6),
         ("band3000_k2", lambda: W.random_band(3000, 9, 100, 11), 2, 3),
         ("convdiff3d_9_k2", lambda: W.conv_diff(9, 3, (50.0, 50.0, 50.0)), 2, 4)]


def run_all(A, k, m, prec, transpose=False):
    rp, ci, av = to_dev(A)
    b, bd = vec(77, A.n)
    S = P.symbolic(rp, ci, k)
    F = P.numeric(S, av)
    ref = oracle.factor(A, k)
    if prec == "ilu":
        pr, kind = F, oracle.PREC_ILU
        Fa = (ref["rowptr"], ref["colind"], ref["val"])
    elif prec == "iilu":
        pr, kind = P.iiluk_build(F), oracle.PREC_IILU
        g = oracle.iiluk_build(A.n, ref["rowptr"], ref["colind"], ref["val"])
        Fa = (ref["rowptr"], ref["colind"], g)
    else:
        pr, kind, Fa = None, oracle.PREC_NONE, None
    out = {}
    for basis in ("store", "recompute", "auto", "minv_vy"):
        x, info = P.gmres(rp, ci, av, bd, pr, restart=m, rtol=1e-10, transpose=transpose,
                          basis=basis)
        out[basis] = (x.clone(), info.iters, info.cycles, info.relres, info.status)
    return out, b, kind, Fa


@pytest.mark.parametrize("name,make,k,m", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", ["ilu", "iilu", "none"])
def test_recompute_bit_identical_to_store_and_oracle(name, make, k, m, prec):
    A = make()
    out, b, kind, Fa = run_all(A, k, m, prec)
    xs, its, cys, rels, sts = out["store"]
    assert sts == 0 and cys >= 2, (sts, cys)  # several restart cycles
    for basis in ("recompute", "auto"):
        x, it, cy, rel, st = out[basis]
        assert (st, it, cy) == (sts, its, cys), basis
        assert bits([rel])[0] == bits([rels])[0], basis
        assert_bits_equal(x, xs, f"{basis} vs store")
    st, xo, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, kind, Fa, m, 1e-10,
                                        dotmode=oracle.DOT_TREE, update=oracle.UPDATE_Z)
    assert (st, it, cyc) == (sts, its, cys)
    assert bits([rel])[0] == bits([rels])[0]
    assert_bits_equal(xs, xo, "store vs oracle")
    # the textbook update against the oracle's textbook mode
    x, it, cy, rel, st = out["minv_vy"]
    st2, xo2, it2, rel2, cyc2 = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, kind, Fa, m,
                                             1e-10, dotmode=oracle.DOT_TREE,
                                             update=oracle.UPDATE_MVY)
    assert (st, it, cy) == (st2, it2, cyc2)
    assert bits([rel])[0] == bits([rel2])[0]
    assert_bits_equal(x, xo2, "minv_vy vs oracle")
    if prec == "none":  # M = I: both cycle ends are the same operations
        assert_bits_equal(x, xs, "minv_vy vs store without preconditioner")


def test_transposed_solve_recompute_bit_identical():
    A = W.conv_diff(16, 2, (20.0, 20.0))
    out, *_ = run_all(A, 2, 5, "ilu", transpose=True)
    xs, its, cys, rels, sts = out["store"]
    assert sts == 0 and cys >= 2
    x, it, cy, rel, st = out["recompute"]
    assert (st, it, cy) == (sts, its, cys) and bits([rel])[0] == bits([rels])[0]
    assert_bits_equal(x, xs, "transposed recompute vs store")


def test_adjoint_gradients_identical_with_recomputed_bases():
    Pt = W.fd_pattern(14, 2)
    n = Pt.n
    theta0 = W.log_uniform(W.stream_key(9, "rb"), np.arange(n), 0.1, 10.0)
    b = W.uniform(W.stream_key(9, "rbb"), np.arange(n), -1.0, 1.0)
    xt = torch.from_numpy(W.uniform(W.stream_key(9, "rbx"), np.arange(n), -1.0, 1.0)).cuda()
    rp = torch.from_numpy(Pt.rowptr).cuda()
    ci = torch.from_numpy(Pt.colind).cuda()
    vals0 = W.fd_values(Pt, torch.from_numpy(theta0), (20.0, 20.0)).cuda()
    grads = {}
    for basis in ("store", "recompute"):
        solver = P.IlukSolver(rp, ci, k=2, restart=8, rtol=1e-12, basis=basis)
        vals = vals0.clone().requires_grad_(True)  # dL/da straight from the adjoint scatter
        bd = torch.from_numpy(b).cuda().requires_grad_(True)
        x = solver.solve(vals, bd)
        ((x - xt) ** 2).sum().backward()
        assert solver.last_forward.cycles >= 2 and solver.last_backward.cycles >= 2
        grads[basis] = (x.detach(), vals.grad, bd.grad)
    for a, c, what in zip(grads["store"], grads["recompute"], ("x", "dL/da", "dL/db")):
        assert_bits_equal(c, a, what)
