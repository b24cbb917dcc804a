"""Inputs against their recipe: the SplitMix64 draws against the generator's
published test values, the random band matrices (columns, values, diagonal
and the 160,000-row headline matrix), the convection-diffusion stencils
against their closed forms, the batched value sets and uneven grids, and the
27-point Poisson matrix (Sec. 4's 3D 27-point central differencing).  Also the
TPILU(k) solve policy of the oracle (Sec. 1: TPIILU first, ILU(k) when it does
not converge) against the plain solves it is made of."""
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


def test_splitmix64_matches_published_outputs():
    """The draws are SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the
    sequence from state s is mix64(s + c * gamma), c = 1, 2, ...  From state
    1234567 its first five outputs are the published test values; from state 0
    the first is 0xE220A8397B1DCDAF."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(v) for v in W.draws_u64(np.uint64(1234567), np.arange(5))] == want
    assert int(W.draws_u64(np.uint64(0), np.arange(1))[0]) == 0xE220A8397B1DCDAF
    # counter-based: a draw depends only on its key and counter
    k = W.stream_key(3, "x")
    assert np.array_equal(W.draws_u64(k, np.array([7, 2])), W.draws_u64(k, np.arange(8))[[7, 2]])
    assert W.stream_key(3, "x") != W.stream_key(3, "y") != W.stream_key(4, "x")


def test_uniform_doubles_have_53_bits_in_range():
    u = W.uniform01(W.stream_key(9, "u"), np.arange(200_000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all((u * 2.0 ** 53) == np.floor(u * 2.0 ** 53))
    assert abs(u.mean() - 0.5) < 0.005
    v = W.log_uniform(W.stream_key(9, "l"), np.arange(200_000), 0.1, 10.0)
    assert v.min() >= 0.1 * (1 - 1e-15) and v.max() < 10.0
    assert abs(np.log(v).mean()) < 0.02  # log-uniform on [log 0.1, log 10]


def check_band(A, noff, hw, rows=None):
    n = A.n
    assert A.nnz == (noff + 1) * n
    assert np.array_equal(A.rowptr, np.arange(0, (noff + 1) * n + 1, noff + 1))
    for i in (range(n) if rows is None else rows):
        cols = A.colind[A.rowptr[i]:A.rowptr[i + 1]].astype(np.int64)
        vals = A.val[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols
        assert cols.min() >= max(0, i - hw) and cols.max() <= min(n - 1, i + hw)
        off = vals[cols != i]
        assert np.all(np.abs(off) <= 1.0) and np.all(off != 0.0)
        s = 0.0
        for v in off:  # the diagonal: 1.2 * sum |a_ij| in column order
            s = s + abs(float(v))
        assert vals[cols == i][0] == 1.2 * s


def test_random_band_recipe():
    A = W.random_band(3000, 9, 200, 7)
    assert A.n == 3000
    check_band(A, 9, 200)
    B = W.random_band(3000, 9, 200, 7)
    assert np.array_equal(A.colind, B.colind) and np.array_equal(A.val, B.val)
    C = W.random_band(3000, 9, 200, 8)
    assert not np.array_equal(A.colind, C.colind)


def test_band_160k_headline_matrix():
    Pb = W.random_band_160k(2)
    A = Pb.A
    assert A.n == 160_000 and A.nnz == 1_600_000
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    d = A.colind.astype(np.int64) - rows
    assert np.abs(d).max() <= 2000
    # offsets uniform over the band without the diagonal: E|d| = 1000.25 away
    # from the edges (interior rows only)
    inner = (rows >= 2000) & (rows < A.n - 2000) & (d != 0)
    assert abs(np.abs(d[inner]).mean() - 1000.25) < 5.0
    assert abs(d[inner].mean()) < 5.0
    edge = list(range(0, 2500)) + list(range(A.n - 2500, A.n))  # rows whose band is clipped
    check_band(A, 9, 2000, edge + list(range(80_000, 81_000)))
    # b = A x* row by row, left to right
    assert np.array_equal(Pb.b, W.matvec_rowseq(A, Pb.xstar))


@pytest.mark.parametrize("d", [2, 3])
def test_conv_diff_closed_form(d):
    """Constant diffusion: the scaled (2d+1)-point Laplacian, 2d on the
    diagonal and -1 to each grid neighbour; first-order upwind convection adds
    h*beta_c to the diagonal and -h*beta_c to the minus-side neighbour."""
    N = 5
    beta = [20.0, 30.0, 50.0][:d]
    h = 1.0 / (N + 1)
    D = W.csr_to_dense(W.conv_diff(N, d, beta))
    n = N ** d
    want = np.zeros((n, n))
    for i in range(n):
        x = [(i // N ** c) % N for c in range(d)]
        diag = 2.0 * d
        for c in range(d):
            diag = diag + h * beta[c]
        want[i, i] = diag
        for c in range(d):
            if x[c] > 0:
                want[i, i - N ** c] = -1.0 - h * beta[c]
            if x[c] < N - 1:
                want[i, i + N ** c] = -1.0
    assert np.array_equal(D, want)


def test_conv_diff_harmonic_faces():
    N = 4
    theta = W.log_uniform(W.stream_key(2, "th"), np.arange(N * N), 0.1, 10.0)
    D = W.csr_to_dense(W.conv_diff(N, 2, (0.0, 0.0), theta))
    for i in range(N * N):
        x, y = i % N, i // N
        for j, inside in ((i - 1, x > 0), (i + 1, x < N - 1), (i - N, y > 0), (i + N, y < N - 1)):
            if inside:
                tp, tq = theta[i], theta[j]
                assert D[i, j] == -(2.0 * tp * tq / (tp + tq))
        # a boundary face takes the cell's own coefficient
        assert np.isclose(D[i].sum(), theta[i] * (4 - sum((x > 0, x < N - 1, y > 0, y < N - 1))),
                          rtol=1e-12, atol=1e-12)


def test_uneven_grids_and_value_sets():
    probs = W.uneven_grids(6, 3, 6)
    assert len(probs) == 6
    for p in probs:
        N = p.extra["side"]
        assert 3 <= N <= 6 and p.A.n == N ** 3 and p.k == 1 and p.restart == 30
        assert np.array_equal(p.b, W.matvec_rowseq(p.A, p.xstar))
    A0, vals, bs, xs = W.batched_values(3, 4)
    assert vals.shape == (3, A0.nnz) and bs.shape == xs.shape == (3, A0.n)
    assert np.array_equal(vals[0], A0.val) and not np.array_equal(vals[0], vals[1])
    for s in range(3):
        A = W.CSR(A0.n, A0.rowptr, A0.colind, vals[s])
        assert np.array_equal(bs[s], W.matvec_rowseq(A, xs[s]))
