"""The sweeps with prefix helpers (ILUK_SCHED_WARP_CLUSTER_HELP) against the
oracle.

A helper cluster publishes, per row, the partial difference over the row's
leading entries whose x is already final; the row's warp continues from it.
The result must not change by a bit, whatever the helpers managed to publish
in time, and a prefix published in one launch must never be taken by a later
one (the launch epoch).  Checked here: single applications on matrices with
long dependency chains and many entries per row (so that helpers do publish),
many applications in a row with different right-hand sides (a prefix left
over from an earlier launch would change the result), both sweep directions
alone and mixed with other schedules, the transposed solve, GMRES and the
one-call solve on the helped schedule, and replays of a CUDA graph that
captured a helped application.
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

HELP = L.SCHED_WARP_CLUSTER_HELP
CASES = [("band20000_k2", W.random_band(20000, 9, 400, 3), 2),
         ("band4000_k3", W.random_band(4000, 9, 200, 5), 3),
         ("convdiff3d_16_k2", W.conv_diff(16, 3, (50.0, 50.0, 50.0)), 2),
         ("rand1000_k2", W.random_sparse(1000, 0.006, 6), 2)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def factored():
    out = {}
    for name, A, k in CASES:
        rp, ci, av = to_dev(A)
        S, F = P.factor(rp, ci, av, k)
        out[name] = (A, k, S, F, oracle.factor(A, k), (rp, ci, av))
    return out


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("width", [384, 512, 1024])
def test_helped_apply_repeated_bit_exact(factored, name, width):
    """Eight applications in a row, each on a new right-hand side, forward
    and transposed: every one equal to the oracle's."""
    A, k, S, F, ref, _ = factored[name]
    sched = L.sched_width(HELP, width)
    trp, tci, tv = oracle.transpose(A.n, ref["rowptr"], ref["colind"], ref["val"])
    for rep in range(8):
        p, pd = vec(100 + rep, A.n)
        y = F.apply(pd, sched=sched)
        assert_bits_equal(y, oracle.apply(A.n, ref["rowptr"], ref["colind"], ref["val"], p),
                          f"{name} apply {rep}")
        if rep % 4 == 3:
            yt = F.apply(pd, transpose=True, sched=sched)
            assert_bits_equal(yt, oracle.apply_t(A.n, trp, tci, tv, p), f"{name} apply_t {rep}")
    assert F.status() == L.OK


@pytest.mark.parametrize("mix", [HELP | (L.SCHED_WARP_CLUSTER << 8),
                                 L.SCHED_WARP_GRID | (HELP << 8),
                                 L.SCHED_FLAGS | (L.sched_width(HELP, 384) << 8)])
def test_helped_sweep_mixed_with_other_schedules(factored, mix):
    A, k, S, F, ref, _ = factored["band20000_k2"]
    for rep in range(3):
        p, pd = vec(200 + rep, A.n)
        assert_bits_equal(F.apply(pd, sched=mix),
                          oracle.apply(A.n, ref["rowptr"], ref["colind"], ref["val"], p),
                          f"mixed {mix:#x} apply {rep}")


def test_helped_gmres_and_one_call_solve(factored):
    A, k, S, F, ref, (rp, ci, av) = factored["band20000_k2"]
    b, bd = vec(300, A.n)
    st, xo, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                                        (ref["rowptr"], ref["colind"], ref["val"]), 10, 1e-10,
                                        dotmode=oracle.DOT_TREE)
    assert st == 0
    F.set_schedule(L.sched_width(HELP, 512))
    x, info = P.gmres(rp, ci, av, bd, F, restart=10, rtol=1e-10)
    assert (info.iters, info.cycles) == (it, cyc) and bits([info.relres])[0] == bits([rel])[0]
    assert_bits_equal(x, xo, "gmres on helped sweeps")
    x2, info2 = P.solve(rp, ci, av, bd, k=k, restart=10, rtol=1e-10,
                        sched=L.sched_width(HELP, 384))
    assert (info2.iters, info2.cycles) == (it, cyc)
    assert_bits_equal(x2, xo, "one-call solve on helped sweeps")


def test_helped_apply_graph_replays(factored):
    """A helped application captured in a CUDA graph and replayed with new
    right-hand sides: the epoch lives on the device, so every replay starts a
    new one and never takes an earlier replay's prefixes."""
    A, k, S, F, ref, _ = factored["band4000_k3"]
    sched = L.sched_width(HELP, 512)
    p0, pd = vec(400, A.n)
    F.apply(pd, sched=sched)  # the helpers' scratch is made outside the capture
    y = torch.empty_like(pd)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.apply(pd, out=y, sched=sched)
    for rep in range(4):
        p, pnew = vec(410 + rep, A.n)
        pd.copy_(pnew)
        g.replay()
        torch.cuda.synchronize()
        assert_bits_equal(y, oracle.apply(A.n, ref["rowptr"], ref["colind"], ref["val"], p),
                          f"replay {rep}")
