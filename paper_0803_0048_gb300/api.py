"""Python binding of libiluk with torch tensors (same names as the C ABI).

PyTorch provides device memory and the current CUDA stream; every step of
the method runs in the library's kernels.  All tensors must live on the
current CUDA device: CSR row pointers int64, column indices int32, values and
vectors float64.  The step labels a1-a8 in the docstrings are those of the
C header (include/iluk.h).
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Tuple

import torch

from . import _lib as L


class IlukError(RuntimeError):
    def __init__(self, status: int, info: Optional[L.Info] = None, what: str = ""):
        lib = L.load()
        msg = lib.iluk_strerror(status).decode()
        row = info.row if info is not None else -1
        super().__init__(f"{what}: {msg} (status {status}, row {row})")
        self.status = status
        self.row = row
        self.info = info


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_dev(*ts):
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda or t.get_device() != torch.cuda.current_device():
            raise ValueError("tensors must be on the current CUDA device")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")


def _vecs(*specs) -> None:
    """Check float64 tensors before their pointers cross the C ABI, which takes
    lengths from the handle or the pattern: the kernels trust dtype and size.
    Each spec is (tensor or None, expected number of elements, name); dtypes and
    sizes of all are checked before devices."""
    for t, n, what in specs:
        if t is None:
            continue
        if t.dtype != torch.float64:
            raise ValueError(f"{what}: expected torch.float64, got {t.dtype}")
        if t.numel() != n:
            raise ValueError(f"{what}: expected {n} elements, got {t.numel()}")
    _check_dev(*(t for t, _, _ in specs))


def _call(fn, *args, info=None, what=""):
    st = fn(*args)
    if st != L.OK:
        raise IlukError(st, info, what or fn.__name__)
    return st


class CsrPattern:
    """A CSR pattern on the device, plus the C struct that points at it."""

    def __init__(self, rowptr: torch.Tensor, colind: torch.Tensor):
        if rowptr.dtype != torch.int64 or colind.dtype != torch.int32:
            raise ValueError("CSR pattern: rowptr must be int64 and colind int32")
        if rowptr.dim() != 1 or colind.dim() != 1 or rowptr.numel() < 1:
            raise ValueError("CSR pattern: rowptr [n+1] and colind [nnz] must be 1-D")
        _check_dev(rowptr, colind)
        self.rowptr, self.colind = rowptr, colind
        self.n = rowptr.numel() - 1
        self.nnz = colind.numel()
        self.c = L.Pattern(self.n, self.nnz, rowptr.data_ptr(), colind.data_ptr())

    @property
    def ref(self):
        return C.byref(self.c)


def validate(rowptr: torch.Tensor, colind: torch.Tensor) -> Tuple[int, int]:
    """a1: returns (status, first bad row)."""
    A = CsrPattern(rowptr, colind)
    info = L.Info()
    st = L.load().iluk_validate(A.ref, C.byref(info), C.c_void_p(_stream()))
    return st, info.row


class Symbolic:
    """Result of the symbolic phase (pattern of F = L~ + U~ and levels).  It
    also keeps, for its pattern, the sweep schedules the autotuner picked on
    the first solve (and on the first transposed solve), which later
    factorizations of the pattern reuse."""

    def __init__(self, handle, A: CsrPattern, k: int):
        self.h = handle
        self.A = A
        self.k = k
        v = L.SymView()
        L.load().iluk_sym_query(self.h, C.byref(v))
        self.n, self.nnz, self.max_row = v.n, v.nnz, v.max_row

    def __del__(self):
        if getattr(self, "h", None):
            torch.cuda.synchronize()
            L.load().iluk_sym_destroy(self.h)
            self.h = None

    def pattern(self):
        """(rowptr int64, colind int32, level uint8, diag int64) device copies."""
        dev = self.A.rowptr.device
        rp = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
        ci = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        lv = torch.empty(self.nnz, dtype=torch.uint8, device=dev)
        dg = torch.empty(self.n, dtype=torch.int64, device=dev)
        _call(L.load().iluk_sym_export, self.h, _ptr(rp), _ptr(ci), _ptr(lv), _ptr(dg),
              C.c_void_p(_stream()))
        return rp, ci, lv, dg

    def depth(self) -> Tuple[int, int]:
        dl, du = C.c_int32(), C.c_int32()
        _call(L.load().iluk_sym_depth, self.h, C.byref(dl), C.byref(du), C.c_void_p(_stream()))
        return dl.value, du.value


def symbolic(rowptr: torch.Tensor, colind: torch.Tensor, k: int) -> Symbolic:
    """a2: symbolic ILU(k) (Algorithm 1 with the levels of Def. 2.3)."""
    A = CsrPattern(rowptr, colind)
    h = C.c_void_p()
    info = L.Info()
    _call(L.load().iluk_symbolic, A.ref, int(k), C.byref(h), C.byref(info),
          C.c_void_p(_stream()), info=info, what="iluk_symbolic")
    return Symbolic(h, A, k)


class Factors:
    """Numeric ILU(k) factors on a symbolic pattern."""

    def __init__(self, handle, S: Symbolic):
        self.h = handle
        self.S = S

    def __del__(self):
        if getattr(self, "h", None):
            torch.cuda.synchronize()
            L.load().iluk_fac_destroy(self.h)
            self.h = None

    def values(self) -> torch.Tensor:
        out = torch.empty(self.S.nnz, dtype=torch.float64, device=self.S.A.rowptr.device)
        _call(L.load().iluk_fac_export, self.h, _ptr(out), C.c_void_p(_stream()))
        return out

    def refactor(self, vals: torch.Tensor) -> None:
        _vecs((vals, self.S.A.nnz, "values of A"))
        info = L.Info()
        _call(L.load().iluk_refactor, self.h, _ptr(vals), C.byref(info), C.c_void_p(_stream()),
              info=info, what="iluk_refactor")

    def apply(self, p: torch.Tensor, out: Optional[torch.Tensor] = None, transpose: bool = False,
              sched: int = L.SCHED_AUTO) -> torch.Tensor:
        """a4: y = (L~U~)^-1 p (or ^-T)."""
        _vecs((p, self.S.n, "p"),
              (out, self.S.n, "out"))
        y = torch.empty_like(p) if out is None else out
        _call(L.load().iluk_apply_sched, self.h, _ptr(p), _ptr(y), int(transpose), int(sched),
              C.c_void_p(_stream()))
        return y

    def status(self) -> int:
        info = L.Info()
        return L.load().iluk_fac_status(self.h, C.byref(info), C.c_void_p(_stream()))

    def set_schedule(self, sched: int) -> None:
        _call(L.load().iluk_set_schedule, self.h, int(sched))

    def schedule(self) -> int:
        return L.load().iluk_get_schedule(self.h)


def numeric(S: Symbolic, vals: torch.Tensor) -> Factors:
    """a3: numeric IKJ factorization (Eq. 1)."""
    _vecs((vals, S.A.nnz, "values of A"))
    h = C.c_void_p()
    info = L.Info()
    _call(L.load().iluk_numeric, S.h, _ptr(vals), C.byref(h), C.byref(info),
          C.c_void_p(_stream()), info=info, what="iluk_numeric")
    return Factors(h, S)


def factor(rowptr: torch.Tensor, colind: torch.Tensor, vals: torch.Tensor, k: int):
    """a2 + a3 with the numeric phase running beside the symbolic one (k >= 2);
    the same (Symbolic, Factors) as ``symbolic`` then ``numeric``, bit for bit.
    The sweeps walk index orders until level orders are built."""
    A = CsrPattern(rowptr, colind)
    _vecs((vals, A.nnz, "values of A"))
    hs, hf = C.c_void_p(), C.c_void_p()
    info = L.Info()
    _call(L.load().iluk_factor, A.ref, _ptr(vals), int(k), C.byref(hs), C.byref(hf),
          C.byref(info), C.c_void_p(_stream()), info=info, what="iluk_factor")
    S = Symbolic(hs, A, k)
    return S, Factors(hf, S)


def solve(rowptr: torch.Tensor, colind: torch.Tensor, vals: torch.Tensor, b: torch.Tensor,
          k: int = 2, restart: int = 30, rtol: float = 1e-8, maxit: int = 10000,
          precond: str = "ilu", check: bool = True, sched: int = 0, x=None,
          return_factors: bool = False):
    """Solve A x = b in one call: the level-k factorization of A (``factor``),
    then right-preconditioned GMRES(restart) from x0 = 0 with the ILU(k) sweeps
    (precond "ilu"), the TPIILU inverses built from the same factors ("iilu"),
    or no preconditioner ("none").  Returns (x, info), plus (Symbolic,
    Factors) with ``return_factors`` (precond "ilu" only).

    With "ilu" this is one C call (iluk_solve): GMRES forms v_1 = b / ||b||
    first, the one-launch factorization (k >= 2) solves L x = v_1 beside its
    numeric phase, and the first preconditioner application runs only its
    backward sweep; the results are those of ``factor`` then ``gmres`` bit
    for bit.  ``sched`` is the sweep schedule (0: autotune once F exists)."""
    if precond not in ("ilu", "iilu", "none"):
        raise ValueError("precond must be 'ilu', 'iilu' or 'none'")
    if return_factors and precond != "ilu":
        raise ValueError("return_factors needs precond 'ilu'")
    if precond == "ilu":
        A = CsrPattern(rowptr, colind)
        _vecs((vals, A.nnz, "values of A"),
              (b, A.n, "b"),
              (x, A.n, "x"))
        xo = torch.empty_like(b) if x is None else x
        hs, hf = C.c_void_p(), C.c_void_p()
        info = L.Info()
        st = L.load().iluk_solve(A.ref, _ptr(vals), int(k), _ptr(b), _ptr(xo), int(restart),
                                 float(rtol), int(maxit), int(sched),
                                 C.byref(hs) if return_factors else None,
                                 C.byref(hf) if return_factors else None, C.byref(info),
                                 C.c_void_p(_stream()))
        facs = None
        if return_factors and hf.value:
            S = Symbolic(hs, A, k)
            facs = (S, Factors(hf, S))
        if check and st != L.OK:
            raise IlukError(st, info, "iluk_solve")
        return (xo, info, facs) if return_factors else (xo, info)
    prec = None
    if precond != "none":
        _, prec = factor(rowptr, colind, vals, k)
        if precond == "iilu":
            prec = iiluk_build(prec)
    return gmres(rowptr, colind, vals, b, prec, restart=restart, rtol=rtol, maxit=maxit,
                 check=check)


class IncompleteInverse:
    """TPIILU level-based incomplete inverses (Sec. 3.5)."""

    def __init__(self, handle, F: Factors):
        self.h = handle
        self.F = F

    def __del__(self):
        if getattr(self, "h", None):
            torch.cuda.synchronize()
            L.load().iiluk_destroy(self.h)
            self.h = None

    def values(self) -> torch.Tensor:
        out = torch.empty(self.F.S.nnz, dtype=torch.float64, device=self.F.S.A.rowptr.device)
        _call(L.load().iiluk_export, self.h, _ptr(out), C.c_void_p(_stream()))
        return out

    def apply(self, p: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        _vecs((p, self.F.S.n, "p"),
              (out, self.F.S.n, "out"))
        y = torch.empty_like(p) if out is None else out
        _call(L.load().iiluk_apply, self.h, _ptr(p), _ptr(y), C.c_void_p(_stream()))
        return y


def iiluk_build(F: Factors) -> IncompleteInverse:
    """a5: build the TPIILU incomplete inverses from the factors."""
    h = C.c_void_p()
    info = L.Info()
    _call(L.load().iiluk_build, F.h, C.byref(h), C.byref(info), C.c_void_p(_stream()),
          info=info, what="iiluk_build")
    return IncompleteInverse(h, F)


def spmv(rowptr, colind, vals, x, out=None):
    A = CsrPattern(rowptr, colind)
    _vecs((vals, A.nnz, "values of A"),
          (x, A.n, "x"),
          (out, A.n, "out"))
    y = torch.empty_like(x) if out is None else out
    _call(L.load().iluk_spmv, A.ref, _ptr(vals), _ptr(x), _ptr(y), C.c_void_p(_stream()))
    return y


def dot(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Fixed-shape inner product (4096 strided partials, pairwise tree)."""
    _vecs((x, x.numel(), "x"),
          (y, x.numel(), "y"))
    out = torch.empty(1, dtype=torch.float64, device=x.device)
    _call(L.load().iluk_dot, x.numel(), _ptr(x), _ptr(y), _ptr(out), C.c_void_p(_stream()))
    return out


def div_rn(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """a / b elementwise by the library's division (integer pipes: a
    fixed-point reciprocal and an exact remainder correction), as the
    numeric phase and the sweeps divide; equal to IEEE division bit for bit."""
    _vecs((a, a.numel(), "a"),
          (b, a.numel(), "b"))
    q = torch.empty_like(a)
    _call(L.load().iluk_div_rn, a.numel(), _ptr(a), _ptr(b), _ptr(q), C.c_void_p(_stream()))
    return q


def gmres(rowptr, colind, vals, b, prec=None, restart=30, rtol=1e-8, maxit=10000,
          transpose=False, x=None, check=True, basis="auto"):
    """a6: right-preconditioned GMRES(m) from x0 = 0.  ``prec`` is None, a
    Factors (ILU(k) sweeps) or an IncompleteInverse (TPIILU).  ``basis``:
    "store" keeps the preconditioned basis and ends a cycle with x += Z y;
    "recompute" keeps only V and applies the preconditioner again at the end
    of a cycle (same bits, less memory); "auto" (default) stores when the
    basis takes at most half of the free device memory; "minv_vy" ends a
    cycle with x += M^-1 (V y).  Returns (x, info)."""
    if basis not in L.BASIS:
        raise ValueError(f"basis must be one of {sorted(L.BASIS)}")
    A = CsrPattern(rowptr, colind)
    _vecs((vals, A.nnz, "values of A"),
          (b, A.n, "b"),
          (x, A.n, "x"))
    xo = torch.empty_like(b) if x is None else x
    if prec is None:
        kind, ph = L.PREC_NONE, None
    elif isinstance(prec, Factors):
        kind, ph = L.PREC_ILU, prec.h
    elif isinstance(prec, IncompleteInverse):
        kind, ph = L.PREC_IILU, prec.h
    else:
        raise TypeError("prec must be None, Factors or IncompleteInverse")
    info = L.Info()
    st = L.load().gmres_solve_ex(A.ref, _ptr(vals), kind, ph, _ptr(b), _ptr(xo), int(restart),
                                 float(rtol), int(maxit), int(transpose), L.BASIS[basis],
                                 C.byref(info), C.c_void_p(_stream()))
    if check and st != L.OK:
        raise IlukError(st, info, "gmres_solve")
    return xo, info


def bicgstab(rowptr, colind, vals, b, prec=None, rtol=1e-8, maxit=10000, x=None, check=True):
    """Right-preconditioned BiCGSTAB from x0 = 0 (the paper's solver, Sec. 4).
    ``prec`` is None, a Factors or an IncompleteInverse.  Returns (x, info);
    info.relres is the true relative residual."""
    A = CsrPattern(rowptr, colind)
    _vecs((vals, A.nnz, "values of A"),
          (b, A.n, "b"),
          (x, A.n, "x"))
    xo = torch.empty_like(b) if x is None else x
    if prec is None:
        kind, ph = L.PREC_NONE, None
    elif isinstance(prec, Factors):
        kind, ph = L.PREC_ILU, prec.h
    elif isinstance(prec, IncompleteInverse):
        kind, ph = L.PREC_IILU, prec.h
    else:
        raise TypeError("prec must be None, Factors or IncompleteInverse")
    info = L.Info()
    st = L.load().bicgstab_solve(A.ref, _ptr(vals), kind, ph, _ptr(b), _ptr(xo), float(rtol),
                                 int(maxit), C.byref(info), C.c_void_p(_stream()))
    if check and st != L.OK:
        raise IlukError(st, info, "bicgstab_solve")
    return xo, info


def tpilu_solve(rowptr, colind, vals, b, F, M=None, solver="gmres", restart=50, rtol=1e-8,
                iilu_maxit=50, maxit=10000, check=True):
    """The TPILU(k) policy (Sec. 1): ``solver`` ("gmres" or "bicgstab") with
    the TPIILU inverses M of F (built when None) for at most ``iilu_maxit``
    iterations, then, if that does not converge, again from x0 = 0 with F's
    ILU(k) sweeps.  Returns (x, info, used) with used "iilu" or "ilu"."""
    A = CsrPattern(rowptr, colind)
    _vecs((vals, A.nnz, "values of A"),
          (b, A.n, "b"))
    xo = torch.empty_like(b)
    kind = {"gmres": L.SOLVER_GMRES, "bicgstab": L.SOLVER_BICGSTAB}[solver]
    info = L.Info()
    used = C.c_int(-1)
    st = L.load().tpilu_solve(A.ref, _ptr(vals), F.h, M.h if M is not None else None, kind,
                              _ptr(b), _ptr(xo), int(restart), float(rtol), int(iilu_maxit),
                              int(maxit), C.byref(used), C.byref(info), C.c_void_p(_stream()))
    if check and st != L.OK:
        raise IlukError(st, info, "tpilu_solve")
    return xo, info, ("iilu" if used.value == L.PREC_IILU else "ilu")


def solve_host(rowptr, colind, vals, b, k, restart=30, rtol=1e-8, maxit=10000, sched=0,
               x=None, check=True):
    """a1-a6 from host memory in one C call (iluk_solve_host): CPU tensors in
    (pinned memory copies fastest), x out on the host.  ``sched`` is a sweep
    schedule (Factors.schedule() of an earlier solve, or 0 to autotune).
    Returns (x, info)."""
    n = rowptr.numel() - 1
    nnz = colind.numel()
    for t, dt, cnt, what in ((rowptr, torch.int64, n + 1, "rowptr"),
                             (colind, torch.int32, nnz, "colind"),
                             (vals, torch.float64, nnz, "values of A"),
                             (b, torch.float64, n, "b"), (x, torch.float64, n, "x")):
        if t is None:
            continue
        if t.device.type != "cpu" or t.dtype != dt or t.numel() != cnt or not t.is_contiguous():
            raise ValueError(f"{what}: need a contiguous host {dt} tensor of {cnt} elements")
    xo = torch.empty(n, dtype=torch.float64, pin_memory=b.is_pinned()) if x is None else x
    info = L.Info()
    st = L.load().iluk_solve_host(n, nnz, _ptr(rowptr), _ptr(colind), _ptr(vals), _ptr(b),
                                  _ptr(xo), int(k), int(restart), float(rtol), int(maxit),
                                  int(sched), C.byref(info), C.c_void_p(_stream()))
    if check and st != L.OK:
        raise IlukError(st, info, "iluk_solve_host")
    return xo, info


def transpose(rowptr, colind, vals):
    """Explicit CSR transpose of A: (rowptr, colind, vals) of A^T on the
    device, columns ascending in each row, values moved exactly."""
    A = CsrPattern(rowptr, colind)
    _vecs((vals, A.nnz, "values of A"))
    trp = torch.empty(A.n + 1, dtype=torch.int64, device=rowptr.device)
    tci = torch.empty(A.nnz, dtype=torch.int32, device=rowptr.device)
    tv = torch.empty(A.nnz, dtype=torch.float64, device=rowptr.device)
    _call(L.load().iluk_transpose, A.ref, _ptr(vals), _ptr(trp), _ptr(tci), _ptr(tv),
          C.c_void_p(_stream()), what="iluk_transpose")
    return trp, tci, tv


def adjoint_scatter(rowptr, colind, lam, x, out=None):
    """gA[p] = -lambda_i x_j on A's pattern."""
    A = CsrPattern(rowptr, colind)
    _vecs((lam, A.n, "lambda"),
          (x, A.n, "x"),
          (out, A.nnz, "out"))
    g = torch.empty(A.nnz, dtype=torch.float64, device=x.device) if out is None else out
    _call(L.load().iluk_adjoint_scatter, A.ref, _ptr(lam), _ptr(x), _ptr(g),
          C.c_void_p(_stream()))
    return g


def numeric_batched(S: Symbolic, vals: torch.Tensor, out: Optional[torch.Tensor] = None):
    """a7: factor ``vals`` [nbatch, nnz_A] on one pattern in one launch.
    Returns (F values [nbatch, nnz_F], per-set statuses)."""
    if vals.dim() != 2:
        raise ValueError("values: expected [nbatch, nnz_A]")
    nb = vals.shape[0]
    _vecs((vals, nb * S.A.nnz, "values [nbatch, nnz_A]"),
          (out, nb * S.nnz, "out [nbatch, nnz_F]"))
    F = torch.empty(nb, S.nnz, dtype=torch.float64, device=vals.device) if out is None else out
    infos = (L.Info * max(nb, 1))()
    L.load().iluk_numeric_batched(S.h, nb, _ptr(vals), _ptr(F), infos, C.c_void_p(_stream()))
    return F, [infos[i].status for i in range(nb)]


def set_wait_limit(ns: int) -> int:
    return L.load().iluk_set_wait_limit(int(ns))


def set_symbolic_variant(variant: int) -> int:
    """The symbolic walk for k <= 1: 0 rows ascending without waits (the
    default), 1 the same last row first, 2 the general walk with waits.  The
    results do not depend on it.  Returns the previous variant."""
    prev = L.load().iluk_set_symbolic_variant(int(variant))
    if prev < 0:
        raise ValueError("variant must be 0, 1 or 2")
    return prev


def debug_hold_row(row: int) -> int:
    return L.load().iluk_debug_hold_row(int(row))


def launch_count() -> int:
    """Kernels launched by libiluk in this process so far."""
    return int(L.load().iluk_launch_count())


def prof_enable(on: bool = True) -> None:
    L.load().iluk_prof_enable(int(on))


def prof_read() -> dict:
    """{kind: (total ms, launches)} for the kernels timed since prof_enable."""
    nk = len(L.PROF_KINDS)
    ms = (C.c_double * nk)()
    cnt = (C.c_int64 * nk)()
    _call(L.load().iluk_prof_read, ms, cnt, nk)
    return {L.PROF_KINDS[k]: (ms[k], cnt[k]) for k in range(nk)}


class BatchSolve:
    """a7: factor + GMRES for many systems in one persistent launch.

    ``items`` is a list of (Symbolic, a_vals, b, x) with device tensors; the
    x tensors receive the solutions.  ``solve()`` only enqueues work (it can be
    captured in a CUDA graph after a first call outside the capture); the
    first call outside a capture times the schedules and keeps the fastest
    (see ``set_schedule``).  The kernel takes the items largest first;
    ``results()`` synchronizes and returns one Info per item, in the order
    of ``items``."""

    def __init__(self, items, restart=30, rtol=1e-8, maxit=10000):
        self.items = list(items)  # keep the tensors alive
        _vecs(*(spec for i, (S, vals, b, x) in enumerate(self.items)
                for spec in ((vals, S.A.nnz, f"item {i}: values of A"),
                             (b, S.n, f"item {i}: b"), (x, S.n, f"item {i}: x"))))
        arr = (L.BatchItem * max(len(self.items), 1))()
        for i, (S, vals, b, x) in enumerate(self.items):
            arr[i] = L.BatchItem(S.h.value if isinstance(S.h, C.c_void_p) else S.h,
                                 S.A.rowptr.data_ptr(), S.A.colind.data_ptr(), vals.data_ptr(),
                                 b.data_ptr(), x.data_ptr())
        self.h = C.c_void_p()
        _call(L.load().iluk_batch_create, arr, len(self.items), int(restart), float(rtol),
              int(maxit), C.byref(self.h), C.c_void_p(_stream()))

    def __del__(self):
        if getattr(self, "h", None):
            torch.cuda.synchronize()
            L.load().iluk_batch_destroy(self.h)
            self.h = None

    def solve(self) -> None:
        _call(L.load().iluk_batch_solve, self.h, C.c_void_p(_stream()))

    def results(self):
        n = len(self.items)
        infos = (L.Info * max(n, 1))()
        L.load().iluk_batch_results(self.h, infos, C.c_void_p(_stream()))
        return [infos[i] for i in range(n)]

    def width(self) -> int:
        return L.load().iluk_batch_width(self.h)

    def spin(self) -> bool:
        """True when the autotuned (or fixed) in-CTA sweeps spin instead of
        ending every level at a barrier."""
        return bool(L.load().iluk_batch_spin(self.h))

    def set_schedule(self, width: int, spin: bool) -> None:
        _call(L.load().iluk_batch_set_schedule, self.h, int(width), int(bool(spin)))
