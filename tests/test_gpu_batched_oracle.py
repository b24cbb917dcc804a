"""a7 batched persistent solve against the oracle.

Each item of a batch is factored (ILU(k), Eq. 1) and solved by
right-preconditioned GMRES(m) inside one persistent launch.  Here every item's
x, iteration count, restart cycles and reported residual are compared bit for
bit with the sequential oracle (oracle.factor + oracle.gmres with the
fixed-tree inner products), item by item, so that the batched kernel is held
to the paper's bit-compatibility promise (Sec. 1) directly and not only
through the single-instance path.

Three batch shapes:
* a small batch (three value sets on one 9^3 pattern and uneven grids of side
  6, 11, 13 and 33, the last one 35,937 rows), under every in-CTA schedule
  (256/512/1024 threads per item, level-barrier or spinning sweeps) and under
  the autotuner's choice;
* the full batched workload (512 value sets on one 32^3 7-point pattern plus
  64 uneven grids with sides in [16, 40]), one launch, of which a seeded
  sample of items, always including the largest grid (40^3 = 64,000 rows)
  and the smallest, is compared with the oracle;
* items of other patterns and levels of fill (k = 1..3) whose rows have more
  pivots or pivot-row entries than the numeric phase's per-warp staging area
  holds, beside rows that fit, under every schedule.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0803_0048_gb300 as P
from paper_0803_0048_gb300 import workloads as W

from gpu_helpers import assert_bits_equal, bits

pytestmark = pytest.mark.gpu

RESTART, RTOL, K = 30, 1e-8, 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def oracle_solve(A: W.CSR, b: np.ndarray, k=K, restart=RESTART, rtol=RTOL):
    F = oracle.factor(A, k)
    return oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                        (F["rowptr"], F["colind"], F["val"]), restart, rtol,
                        dotmode=oracle.DOT_TREE)


def check_item(A: W.CSR, b: np.ndarray, x: torch.Tensor, r, what: str):
    st, xo, it, rel, cyc = oracle_solve(A, b)
    assert st == 0, f"{what}: oracle status {st}"
    assert r.status == 0, f"{what}: batched status {r.status} at row {r.row}"
    assert (r.iters, r.cycles) == (it, cyc), f"{what}: iterations {(r.iters, r.cycles)} vs {(it, cyc)}"
    assert bits([r.relres])[0] == bits([rel])[0], f"{what}: relres {r.relres!r} vs {rel!r}"
    assert_bits_equal(x, xo, f"{what}: x")


def fd_instance(N, seed):
    Pt = W.fd_pattern(N, 3)
    th = W.log_uniform(W.stream_key(seed, "bo.theta"), np.arange(Pt.n), 0.1, 10.0)
    beta = W.uniform(W.stream_key(seed, "bo.beta"), np.arange(3), 0.0, 30.0)
    vals = W.fd_values(Pt, torch.from_numpy(th), [float(v) for v in beta]).numpy()
    b = W.uniform(W.stream_key(seed, "bo.rhs"), np.arange(Pt.n), -1.0, 1.0)
    return Pt, vals, b


def small_batch():
    """Three value sets on one 9^3 pattern, then grids of side 6, 11, 13, 33."""
    dev = torch.device("cuda")
    items, host = [], []
    shared = W.fd_pattern(9, 3)
    rp = torch.from_numpy(shared.rowptr).to(dev)
    ci = torch.from_numpy(shared.colind).to(dev)
    S = P.symbolic(rp, ci, K)
    for s in range(3):
        _, vals, b = fd_instance(9, 300 + s)
        items.append((S, torch.from_numpy(vals).to(dev), torch.from_numpy(b).to(dev),
                      torch.empty(shared.n, dtype=torch.float64, device=dev)))
        host.append((W.CSR(shared.n, shared.rowptr, shared.colind, vals), b))
    for N in (6, 11, 13, 33):
        Pt, vals, b = fd_instance(N, 400 + N)
        r = torch.from_numpy(Pt.rowptr).to(dev)
        c = torch.from_numpy(Pt.colind).to(dev)
        items.append((P.symbolic(r, c, K), torch.from_numpy(vals).to(dev),
                      torch.from_numpy(b).to(dev),
                      torch.empty(Pt.n, dtype=torch.float64, device=dev)))
        host.append((W.CSR(Pt.n, Pt.rowptr, Pt.colind, vals), b))
    return items, host


@pytest.fixture(scope="module")
def small():
    items, host = small_batch()
    ref = [oracle_solve(A, b) for A, b in host]
    return items, host, ref


@pytest.mark.parametrize("sched", ["auto", (256, False), (256, True), (512, False), (512, True),
                                   (1024, False), (1024, True)],
                         ids=["auto", "256-level", "256-spin", "512-level", "512-spin", "1024-level",
                              "1024-spin"])
def test_batched_items_bit_exact_vs_oracle(small, sched):
    items, host, ref = small
    for _, _, _, x in items:
        x.fill_(float("nan"))
    B = P.BatchSolve(items, restart=RESTART, rtol=RTOL)
    if sched != "auto":
        B.set_schedule(*sched)
    B.solve()
    res = B.results()
    if sched != "auto":
        assert (B.width(), B.spin()) == sched
    for i, ((_, _, _, x), (A, b), r, (st, xo, it, rel, cyc)) in enumerate(zip(items, host, res, ref)):
        assert st == 0 and r.status == 0, (i, r.status, st)
        assert (r.iters, r.cycles) == (it, cyc), (i, r.iters, it)
        assert bits([r.relres])[0] == bits([rel])[0], (i, r.relres, rel)
        assert_bits_equal(x, xo, f"item {i} (n={A.n}) x")


def test_full_batched_workload_sampled_items_vs_oracle():
    """512 x 32^3 value sets + 64 uneven grids 16^3-40^3, one launch; a seeded
    sample of 12 value sets and 8 grids (the largest and smallest included)
    against the oracle bit for bit; every item converged."""
    dev = torch.device("cuda")
    A0, vals, bs, _ = W.batched_values(512, 32)
    grids = W.uneven_grids(64)
    rp = torch.from_numpy(A0.rowptr).to(dev)
    ci = torch.from_numpy(A0.colind).to(dev)
    S0 = P.symbolic(rp, ci, K)
    items = []
    for s in range(vals.shape[0]):
        items.append((S0, torch.from_numpy(vals[s]).to(dev), torch.from_numpy(bs[s]).to(dev),
                      torch.empty(A0.n, dtype=torch.float64, device=dev)))
    for g in grids:
        r = torch.from_numpy(g.A.rowptr).to(dev)
        c = torch.from_numpy(g.A.colind).to(dev)
        items.append((P.symbolic(r, c, K), torch.from_numpy(g.A.val).to(dev),
                      torch.from_numpy(g.b).to(dev),
                      torch.empty(g.A.n, dtype=torch.float64, device=dev)))
    B = P.BatchSolve(items, restart=RESTART, rtol=RTOL)
    B.solve()
    res = B.results()
    assert all(r.status == 0 for r in res), [i for i, r in enumerate(res) if r.status != 0][:8]
    rng = np.random.default_rng(0x5EED0004)
    sets = sorted(rng.choice(vals.shape[0], size=12, replace=False).tolist())
    sizes = np.array([g.A.n for g in grids])
    largest, smallest = int(np.argmax(sizes)), int(np.argmin(sizes))
    assert sizes[largest] == 40 ** 3
    others = [g for g in rng.permutation(len(grids)).tolist() if g not in (largest, smallest)]
    gsel = sorted({largest, smallest, *others[:6]})
    for s in sets:
        A = W.CSR(A0.n, A0.rowptr, A0.colind, vals[s])
        check_item(A, bs[s], items[s][3], res[s], f"value set {s}")
    for g in gsel:
        i = vals.shape[0] + g
        check_item(grids[g].A, grids[g].b, items[i][3], res[i],
                   f"grid {g} (side {round(grids[g].A.n ** (1 / 3))})")


def mixed_k_batch():
    """Items whose rows have more pivots, or more pivot-row entries, than a
    warp's staging area of the numeric phase holds at some or all CTA widths
    (so those rows take the pivot-by-pivot path), beside rows that fit:
    a random band matrix at k = 3 (up to 60 pivots, 2,884 pivot entries),
    the 27-point Poisson matrix at k = 1 (31 pivots), a 7-point grid at k = 2
    (11 pivots, 121 entries) and a random sparse matrix at k = 3 (rows of up
    to 307 entries)."""
    dev = torch.device("cuda")
    cases = [(W.random_band(600, 9, 60, 21), 3), (W.poisson27(8), 1),
             (W.conv_diff(10, 3, (20.0, 20.0, 20.0)), 2), (W.random_sparse(400, 0.02, 9), 3)]
    items, host = [], []
    for A, k in cases:
        b = W.uniform(W.stream_key(77, f"mixed.rhs.{A.n}"), np.arange(A.n), -1.0, 1.0)
        r = torch.from_numpy(A.rowptr).to(dev)
        c = torch.from_numpy(A.colind).to(dev)
        items.append((P.symbolic(r, c, k), torch.from_numpy(A.val).to(dev),
                      torch.from_numpy(b).to(dev), torch.empty(A.n, dtype=torch.float64, device=dev)))
        host.append((A, b, k))
    return items, host


@pytest.fixture(scope="module")
def mixed():
    items, host = mixed_k_batch()
    ref = [oracle_solve(A, b, k=k) for A, b, k in host]
    return items, host, ref


@pytest.mark.parametrize("sched", [(256, False), (256, True), (512, False), (512, True),
                                   (1024, False), (1024, True)],
                         ids=["256-level", "256-spin", "512-level", "512-spin", "1024-level",
                              "1024-spin"])
def test_batched_long_rows_bit_exact_vs_oracle(mixed, sched):
    items, host, ref = mixed
    for _, _, _, x in items:
        x.fill_(float("nan"))
    B = P.BatchSolve(items, restart=RESTART, rtol=RTOL)
    B.set_schedule(*sched)
    B.solve()
    res = B.results()
    for i, ((_, _, _, x), (A, b, k), r, (st, xo, it, rel, cyc)) in enumerate(
            zip(items, host, res, ref)):
        assert st == 0 and r.status == 0, (i, r.status, st)
        assert (r.iters, r.cycles) == (it, cyc), (i, r.iters, it)
        assert bits([r.relres])[0] == bits([rel])[0], (i, r.relres, rel)
        assert_bits_equal(x, xo, f"item {i} (n={A.n}, k={k}) x")
