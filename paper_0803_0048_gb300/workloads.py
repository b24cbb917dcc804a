"""Seeded synthetic inputs for ILU(k)-preconditioned solves of sparse Ax = b.

This module only *builds* inputs: sparsity patterns, matrix values, right-hand
sides and parameters.  It contains none of the ILU(k) / GMRES arithmetic, so
both the CUDA path and the CPU oracle can consume the same bytes.

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): draw number
``c`` of a stream with key ``s`` is ``mix64(s + (c + 1) * 0x9E3779B97F4A7C15)``,
and a uniform double in [0, 1) is ``(draw >> 11) * 2**-53``.  Because every
draw is a pure function of (key, counter), the inputs are bit-identical on any
machine and independent of vectorisation.

Workloads (all CSR, 0-based, int64 row pointers, int32 sorted unique columns,
float64 values):

* ``conv_diff``: d-dimensional (d = 2 or 3) convection-diffusion
  -div(theta grad u) + beta . grad u on an N^d interior grid, h = 1/(N+1),
  natural lexicographic ordering with x fastest, zero Dirichlet boundary,
  scaled by h^2.  Diffusion faces use the harmonic mean of the two cell
  coefficients (the cell's own value at a boundary face); convection is
  first-order upwind for beta >= 0, which adds h*beta_c to the diagonal and
  -h*beta_c to the upstream (minus-side) neighbour.
* ``random_band``: n rows, each with ``noff`` distinct off-diagonal columns drawn
  uniformly without replacement from the band |j - i| <= halfwidth, values
  uniform in [-1, 1], diagonal 1.2 * sum |a_ij| (summed in column order).
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASTER_SEED = 0x5EED0000


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, tag: str) -> np.uint64:
    """Key of the named stream ``tag`` under master ``seed``."""
    h = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    for ch in tag.encode():
        h = _mix64(h ^ np.uint64(ch))
    return _mix64(h)[0]


def draws_u64(key: np.uint64, counters: np.ndarray) -> np.ndarray:
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + (c + np.uint64(1)) * _GAMMA)


def uniform01(key: np.uint64, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (draws_u64(key, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(key: np.uint64, counters: np.ndarray, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform01(key, counters)


def log_uniform(key: np.uint64, counters: np.ndarray, lo: float, hi: float) -> np.ndarray:
    return np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * uniform01(key, counters))


@dataclasses.dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int64[n+1]
    colind: np.ndarray  # int32[nnz]
    val: np.ndarray     # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def matvec_rowseq(A: CSR, x: np.ndarray) -> np.ndarray:
    """b = A x with every row summed left to right, one rounding per step.

    Used only to make right-hand sides b = A x* for the synthetic problems.
    """
    deg = np.diff(A.rowptr)
    acc = np.zeros(A.n, dtype=np.float64)
    start = A.rowptr[:-1]
    for p in range(int(deg.max(initial=0))):
        rows = np.nonzero(deg > p)[0]
        q = start[rows] + p
        prod = A.val[q] * x[A.colind[q]]
        acc[rows] = acc[rows] + prod
    return acc


# ---------------------------------------------------------------------------
# Finite-difference convection-diffusion on an N^d grid
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class FDPattern:
    """CSR pattern of a (2d+1)-point stencil plus the slot map.

    ``slot[s]`` gives, for every cell, the CSR position of stencil slot ``s``
    (-1 where that neighbour is outside the grid).  Slots are ordered like the
    sorted columns: minus-side neighbours from the slowest dimension to the
    fastest, the diagonal, then plus-side neighbours from fastest to slowest.
    """
    N: int
    d: int
    rowptr: np.ndarray
    colind: np.ndarray
    slot: np.ndarray          # int64[2d+1, n]
    minus_slot: list          # per dimension c (0 = x): slot index
    plus_slot: list
    diag_slot: int

    @property
    def n(self) -> int:
        return self.N ** self.d


def fd_pattern(N: int, d: int) -> FDPattern:
    n = N ** d
    idx = np.arange(n, dtype=np.int64)
    coords = [(idx // (N ** c)) % N for c in range(d)]  # c = 0 is x (fastest)
    strides = [N ** c for c in range(d)]
    # sorted column order: -z, -y, -x, diag, +x, +y, +z
    order = []
    for c in reversed(range(d)):
        order.append(("m", c))
    order.append(("d", -1))
    for c in range(d):
        order.append(("p", c))
    present = []
    cols = []
    for kind, c in order:
        if kind == "d":
            present.append(np.ones(n, dtype=bool))
            cols.append(idx)
        elif kind == "m":
            present.append(coords[c] > 0)
            cols.append(idx - strides[c])
        else:
            present.append(coords[c] < N - 1)
            cols.append(idx + strides[c])
    present = np.stack(present)           # [S, n]
    cols = np.stack(cols)
    deg = present.sum(axis=0)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=rowptr[1:])
    # position of slot s in row i = rowptr[i] + number of present slots before s
    before = np.cumsum(present, axis=0) - present
    slot = np.where(present, rowptr[:-1][None, :] + before, -1).astype(np.int64)
    colind = np.empty(int(rowptr[-1]), dtype=np.int32)
    for s in range(len(order)):
        m = present[s]
        colind[slot[s, m]] = cols[s, m]
    minus_slot = [None] * d
    plus_slot = [None] * d
    diag_slot = None
    for s, (kind, c) in enumerate(order):
        if kind == "m":
            minus_slot[c] = s
        elif kind == "p":
            plus_slot[c] = s
        else:
            diag_slot = s
    return FDPattern(N, d, rowptr, colind, slot, minus_slot, plus_slot, diag_slot)


def fd_values(P: FDPattern, theta: Optional[torch.Tensor], beta: Sequence[float]) -> torch.Tensor:
    """Values of the scaled convection-diffusion matrix on pattern ``P``.

    Written with differentiable torch float64 ops so that the same function
    gives A(theta) for gradient computations.  ``theta`` is a per-cell
    diffusion coefficient (None means 1 everywhere); ``beta`` the constant
    velocity (components >= 0).
    """
    N, d, n = P.N, P.d, P.n
    h = 1.0 / (N + 1)
    for b in beta:
        if b < 0:
            raise ValueError("upwind assembly here expects beta >= 0")
    if theta is None:
        theta = torch.ones(n, dtype=torch.float64)
    dev = theta.device
    idx = torch.arange(n, dtype=torch.int64, device=dev)
    nnz = int(P.rowptr[-1])
    slot = torch.from_numpy(P.slot).to(dev)
    diag = torch.zeros(n, dtype=torch.float64, device=dev)
    val = torch.zeros(nnz, dtype=torch.float64, device=dev)
    for c in range(d):
        stride = N ** c
        coord = (idx // stride) % N
        for side in (-1, +1):
            inside = (coord > 0) if side < 0 else (coord < N - 1)
            nb = torch.clamp(idx + side * stride, 0, n - 1)
            tP, tQ = theta, theta[nb]
            kf = torch.where(inside, 2.0 * tP * tQ / (tP + tQ), tP)
            diag = diag + kf
            s = P.minus_slot[c] if side < 0 else P.plus_slot[c]
            pos = slot[s][inside]
            off = -kf[inside]
            if side < 0:
                off = off - h * float(beta[c])
            val = val.index_put((pos,), off)
    for c in range(d):
        diag = diag + h * float(beta[c])
    val = val.index_put((slot[P.diag_slot],), diag)
    return val


def conv_diff(N: int, d: int, beta: Sequence[float], theta: Optional[np.ndarray] = None) -> CSR:
    P = fd_pattern(N, d)
    th = None if theta is None else torch.from_numpy(np.ascontiguousarray(theta, dtype=np.float64))
    val = fd_values(P, th, beta).numpy()
    return CSR(P.n, P.rowptr, P.colind, np.ascontiguousarray(val))


# ---------------------------------------------------------------------------
# Random banded diagonally dominant matrix
# ---------------------------------------------------------------------------
def random_band(n: int, noff: int, halfwidth: int, seed: int) -> CSR:
    kc = stream_key(seed, "band.cols")
    kv = stream_key(seed, "band.vals")
    rows = np.arange(n, dtype=np.int64)
    lo = np.maximum(0, rows - halfwidth)
    hi = np.minimum(n - 1, rows + halfwidth)
    width = hi - lo + 1
    if int((width - 1).min()) < noff:
        raise ValueError("band too narrow for the requested off-diagonals")
    MAXDRAW = 256
    chosen = np.full((n, noff), -1, dtype=np.int64)
    count = np.zeros(n, dtype=np.int64)
    draw = np.zeros(n, dtype=np.int64)
    todo = rows.copy()
    while todo.size:
        if int(draw[todo].max()) >= MAXDRAW:
            raise RuntimeError("column sampling did not finish")
        u = uniform01(kc, todo * MAXDRAW + draw[todo])
        draw[todo] += 1
        c = lo[todo] + np.floor(u * width[todo]).astype(np.int64)
        dup = (chosen[todo] == c[:, None]).any(axis=1) | (c == todo)
        acc = todo[~dup]
        chosen[acc, count[acc]] = c[~dup]
        count[acc] += 1
        todo = todo[count[todo] < noff]
    chosen.sort(axis=1)
    # off-diagonal values uniform in [-1, 1], redrawing an exact zero
    MAXV = 8
    vals = np.zeros((n, noff), dtype=np.float64)
    vcount = np.zeros((n, noff), dtype=np.int64)
    need = np.ones((n, noff), dtype=bool)
    base = (rows[:, None] * noff + np.arange(noff)[None, :]) * MAXV
    while need.any():
        r, s = np.nonzero(need)
        v = uniform(kv, base[r, s] + vcount[r, s], -1.0, 1.0)
        vcount[r, s] += 1
        vals[r, s] = v
        need[r, s] = v == 0.0
    dsum = np.zeros(n, dtype=np.float64)
    for s in range(noff):
        dsum = dsum + np.abs(vals[:, s])
    dval = 1.2 * dsum
    # merge the diagonal into the sorted columns
    cols = np.concatenate([chosen, rows[:, None]], axis=1)
    allv = np.concatenate([vals, dval[:, None]], axis=1)
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    allv = np.take_along_axis(allv, order, axis=1)
    rowptr = np.arange(0, n * (noff + 1) + 1, noff + 1, dtype=np.int64)
    return CSR(n, rowptr, cols.reshape(-1).astype(np.int32), allv.reshape(-1).copy())


# ---------------------------------------------------------------------------
# The named synthetic problems
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    name: str
    A: CSR
    b: np.ndarray
    xstar: np.ndarray
    k: int
    restart: int
    rtol: float
    extra: dict = dataclasses.field(default_factory=dict)


def _xstar(seed: int, n: int) -> np.ndarray:
    return uniform(stream_key(seed, "xstar"), np.arange(n), -1.0, 1.0)


def conv_diff_2d_64(k: int = 2) -> Problem:
    """2D upwind convection-diffusion, 64x64 interior grid, beta = (20, 20)."""
    seed = MASTER_SEED + 1
    A = conv_diff(64, 2, (20.0, 20.0))
    xs = _xstar(seed, A.n)
    return Problem("convdiff2d_64x64", A, matvec_rowseq(A, xs), xs, k, 30, 1e-8)


def random_band_160k(k: int = 2, n: int = 160_000) -> Problem:
    """n = 160,000, 9 off-diagonals per row within |j - i| <= 2000."""
    seed = MASTER_SEED + 2
    A = random_band(n, 9, 2000, seed)
    xs = _xstar(seed, A.n)
    return Problem(f"random_band_n{n}", A, matvec_rowseq(A, xs), xs, k, 50, 1e-8)


def conv_diff_3d(N: int = 64, k: int = 2, beta=(50.0, 50.0, 50.0)) -> Problem:
    """3D upwind convection-diffusion, N^3 interior grid, beta = (50, 50, 50)."""
    seed = MASTER_SEED + 3
    A = conv_diff(N, 3, beta)
    xs = _xstar(seed, A.n)
    return Problem(f"convdiff3d_{N}^3", A, matvec_rowseq(A, xs), xs, k, 50, 1e-8)


def poisson27(N: int) -> CSR:
    """Poisson's equation on an N^3 interior grid by 27-point central
    differencing (the paper's Sec. 4 workload, grids 50^3 to 90^3): 26 on the
    diagonal and -1 for each of the 26 neighbours (face, edge and corner)
    inside the grid; zero Dirichlet boundary; natural ordering, x fastest.
    Columns are emitted in ascending order."""
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % N, (idx // N) % N, idx // (N * N)
    cols, vals = [], []
    # offsets in ascending column order: dz outermost, then dy, then dx
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                ok = ((x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N) &
                      (z + dz >= 0) & (z + dz < N))
                c = np.where(ok, idx + dx + N * dy + N * N * dz, -1)
                v = 26.0 if (dx, dy, dz) == (0, 0, 0) else -1.0
                cols.append(c)
                vals.append(np.full(n, v))
    C = np.stack(cols, axis=1)
    V = np.stack(vals, axis=1)
    keep = C >= 0
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(keep.sum(axis=1))
    return CSR(n, rowptr, C[keep].astype(np.int32), V[keep].astype(np.float64))


def poisson27_problem(N: int = 50, k: int = 0) -> Problem:
    """27-point Poisson on an N^3 grid, b = A x* for a uniform x*, GMRES(50)."""
    seed = MASTER_SEED + 6
    A = poisson27(N)
    xs = _xstar(seed, A.n)
    return Problem(f"poisson27_{N}^3", A, matvec_rowseq(A, xs), xs, k, 50, 1e-8)


def batched_values(nsets: int = 512, N: int = 32, seed: int = MASTER_SEED + 4):
    """``nsets`` value sets on one N^3 7-point pattern.

    Per set: per-cell diffusion log-uniform in [0.1, 10], beta uniform in
    [0, 30]^3.  Returns (pattern CSR with the first set's values, values
    [nsets, nnz], b [nsets, n], xstar [nsets, n]).
    """
    P = fd_pattern(N, 3)
    n = P.n
    kt = stream_key(seed, "batch.theta")
    kb = stream_key(seed, "batch.beta")
    kx = stream_key(seed, "batch.xstar")
    vals, bs, xs = [], [], []
    for s in range(nsets):
        theta = log_uniform(kt, s * n + np.arange(n), 0.1, 10.0)
        beta = uniform(kb, s * 3 + np.arange(3), 0.0, 30.0)
        v = fd_values(P, torch.from_numpy(theta), [float(x) for x in beta]).numpy()
        A = CSR(n, P.rowptr, P.colind, v)
        x = uniform(kx, s * n + np.arange(n), -1.0, 1.0)
        vals.append(v)
        xs.append(x)
        bs.append(matvec_rowseq(A, x))
    A0 = CSR(n, P.rowptr, P.colind, vals[0])
    return A0, np.stack(vals), np.stack(bs), np.stack(xs)


def uneven_grids(ngrids: int = 64, lo: int = 16, hi: int = 40, seed: int = MASTER_SEED + 4):
    """``ngrids`` 3D problems with sides drawn uniformly from [lo, hi]."""
    kside = stream_key(seed, "uneven.side")
    kt = stream_key(seed, "uneven.theta")
    kb = stream_key(seed, "uneven.beta")
    kx = stream_key(seed, "uneven.xstar")
    sides = lo + np.floor(uniform01(kside, np.arange(ngrids)) * (hi - lo + 1)).astype(np.int64)
    probs = []
    for g, N in enumerate(sides):
        N = int(N)
        n = N ** 3
        theta = log_uniform(kt, g * hi ** 3 + np.arange(n), 0.1, 10.0)
        beta = uniform(kb, g * 3 + np.arange(3), 0.0, 30.0)
        A = conv_diff(N, 3, [float(x) for x in beta], theta)
        x = uniform(kx, g * hi ** 3 + np.arange(n), -1.0, 1.0)
        probs.append(Problem(f"uneven_{g}_{N}^3", A, matvec_rowseq(A, x), x, 1, 30, 1e-8,
                             {"side": N}))
    return probs


def adjoint_problem(N: int = 256):
    """2D diffusion-convection with per-cell diffusion theta, beta = (20, 20).

    Returns (pattern, theta, beta, b, x_target).  b = A(theta) x* for a
    uniform x*; x_target is an independent uniform vector.
    """
    seed = MASTER_SEED + 5
    P = fd_pattern(N, 2)
    n = P.n
    theta = log_uniform(stream_key(seed, "adj.theta"), np.arange(n), 0.1, 10.0)
    beta = (20.0, 20.0)
    v = fd_values(P, torch.from_numpy(theta), beta).numpy()
    A = CSR(n, P.rowptr, P.colind, v)
    xs = _xstar(seed, n)
    xt = uniform(stream_key(seed, "adj.xtarget"), np.arange(n), -1.0, 1.0)
    return P, theta, beta, matvec_rowseq(A, xs), xt


# ---------------------------------------------------------------------------
# Small random cases for parity tests
# ---------------------------------------------------------------------------
def random_sparse(n: int, density: float, seed: int, diag: bool = True,
                  dominance: Optional[float] = 1.5, symmetric_pattern: bool = False) -> CSR:
    """A small random sparse matrix (pattern density ``density``).

    With ``dominance`` set, the diagonal is dominance * sum|offdiag| (+1 for
    empty rows); with None, diagonal values are uniform like the rest.
    """
    key_p = stream_key(seed, "rs.pattern")
    key_v = stream_key(seed, "rs.vals")
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u = uniform01(key_p, (ii * n + jj).reshape(-1)).reshape(n, n)
    mask = u < density
    if symmetric_pattern:
        mask = mask | mask.T
    np.fill_diagonal(mask, diag)
    vals = uniform(key_v, (ii * n + jj).reshape(-1), -1.0, 1.0).reshape(n, n)
    vals[vals == 0.0] = 0.5
    vals = np.where(mask, vals, 0.0)
    if diag and dominance is not None:
        off = np.abs(vals).sum(axis=1) - np.abs(np.diag(vals))
        np.fill_diagonal(vals, dominance * off + 1.0)
    return dense_to_csr(vals, mask)


def dense_to_csr(vals: np.ndarray, mask: Optional[np.ndarray] = None) -> CSR:
    if mask is None:
        mask = vals != 0.0
    n = vals.shape[0]
    deg = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=rowptr[1:])
    r, c = np.nonzero(mask)
    return CSR(n, rowptr, c.astype(np.int32), vals[r, c].astype(np.float64))


def csr_to_dense(A: CSR) -> np.ndarray:
    D = np.zeros((A.n, A.n))
    r = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    D[r, A.colind] = A.val
    return D
