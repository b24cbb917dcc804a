"""The oracle: a sequential FP64 CPU statement of ILU(k) + GMRES.

TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the benchmark's CPU
baseline call it to check or time the CUDA library; the library itself never
imports, links or calls anything here.

The arithmetic lives in ``iluk_oracle.c`` (compiled with ``-O2
-ffp-contract=off``, no fast-math); this module compiles it on first use and
wraps it with ctypes and numpy arrays.  Each wrapper names the part of the
paper it restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iluk_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EPATTERN, ENODIAG, EZEROPIVOT, ENONFINITE, ENOMEM, ENOCONV = 0, 1, 2, 3, 4, 5, 6, 8
PREC_NONE, PREC_ILU, PREC_IILU = 0, 1, 2
DOT_SEQ, DOT_TREE = 0, 1
UPDATE_Z, UPDATE_MVY = 0, 1  # how a GMRES cycle ends: x += Z y, or x += M^-1 (V y)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain gcc, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                        "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        i64, i32 = C.c_int64, C.c_int
        lib.orc_check_pattern.argtypes = [i64, P, P, P]
        lib.orc_symbolic.argtypes = [i64, P, P, i32]
        lib.orc_symbolic.restype = P
        lib.orc_sym_status.argtypes = [P, P, P]
        lib.orc_sym_copy.argtypes = [P, P, P, P]
        lib.orc_sym_free.argtypes = [P]
        lib.orc_numeric.argtypes = [i64, P, P, P, P, P, P, P]
        for f in ("orc_lsolve", "orc_usolve", "orc_apply", "orc_apply_t", "orc_iiluk_apply"):
            getattr(lib, f).argtypes = [i64, P, P, P, P, P]
        lib.orc_iiluk_build.argtypes = [i64, P, P, P, P]
        lib.orc_transpose.argtypes = [i64, P, P, P, P, P, P]
        lib.orc_dot.argtypes = [i64, P, P, i32]
        lib.orc_dot.restype = C.c_double
        lib.orc_spmv.argtypes = [i64, P, P, P, P, P]
        lib.orc_gmres.argtypes = [i64, P, P, P, i32, i32, P, P, P, P, P, i32, C.c_double, i32,
                                  i32, P]
        lib.orc_gmres_update.argtypes = [i64, P, P, P, i32, i32, P, P, P, P, P, i32, C.c_double,
                                         i32, i32, i32, P]
        lib.orc_adjoint.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, i32, C.c_double, i32,
                                    i32, P]
        lib.orc_bicgstab.argtypes = [i64, P, P, P, i32, P, P, P, P, P, C.c_double, i32, i32, P]
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    def __init__(self, status: int, row: int, what: str):
        super().__init__(f"{what}: status {status} at row {row}")
        self.status = status
        self.row = row


def check_pattern(n, rowptr, colind):
    lib = _load()
    rp, ci = _i64(rowptr), _i32(colind)
    bad = np.zeros(1, dtype=np.int64)
    st = lib.orc_check_pattern(n, _p(rp), _p(ci), _p(bad))
    return st, int(bad[0])


def symbolic(n, rowptr, colind, k):
    """Algorithm 1 (Sec. 2.2) with the level of Def. 2.3.

    Returns (status, bad_row, F_rowptr, F_colind, F_level)."""
    lib = _load()
    rp, ci = _i64(rowptr), _i32(colind)
    h = lib.orc_symbolic(n, _p(rp), _p(ci), int(k))
    try:
        bad = np.zeros(1, dtype=np.int64)
        nnz = np.zeros(1, dtype=np.int64)
        st = lib.orc_sym_status(h, _p(bad), _p(nnz))
        if st in (EINVAL, EPATTERN):
            return st, int(bad[0]), None, None, None
        frp = np.zeros(n + 1, dtype=np.int64)
        fci = np.zeros(max(int(nnz[0]), 1), dtype=np.int32)
        flev = np.zeros(max(int(nnz[0]), 1), dtype=np.uint8)
        lib.orc_sym_copy(h, _p(frp), _p(fci), _p(flev))
        nn = int(nnz[0])
        return st, int(bad[0]), frp, fci[:nn].copy(), flev[:nn].copy()
    finally:
        lib.orc_sym_free(h)


def numeric(n, arp, aci, av, frp, fci):
    """IKJ numeric factorization (Eq. 1, Eqs. lufactor2/lufactor).

    Returns (status, bad_row, F_val)."""
    lib = _load()
    arp, aci, av = _i64(arp), _i32(aci), _f64(av)
    frp, fci = _i64(frp), _i32(fci)
    fv = np.zeros(max(int(frp[-1]), 1), dtype=np.float64)
    bad = np.zeros(1, dtype=np.int64)
    st = lib.orc_numeric(n, _p(arp), _p(aci), _p(av), _p(frp), _p(fci), _p(fv), _p(bad))
    return st, int(bad[0]), fv[: int(frp[-1])].copy()


def _vec_call(fname, n, rp, ci, v, p):
    lib = _load()
    rp, ci, v, p = _i64(rp), _i32(ci), _f64(v), _f64(p)
    y = np.zeros(max(n, 1), dtype=np.float64)
    getattr(lib, fname)(n, _p(rp), _p(ci), _p(v), _p(p), _p(y))
    return y[:n].copy()


def lsolve(n, frp, fci, fv, p):
    """Forward sweep, Eq. forwardsubA."""
    return _vec_call("orc_lsolve", n, frp, fci, fv, p)


def usolve(n, frp, fci, fv, x):
    """Backward sweep with U~, each row right to left, divide by u_ii last."""
    return _vec_call("orc_usolve", n, frp, fci, fv, x)


def apply(n, frp, fci, fv, p):
    """y = (L~U~)^-1 p by the two sweeps (Eq. triangleSolve)."""
    return _vec_call("orc_apply", n, frp, fci, fv, p)


def transpose(n, rp, ci, v=None):
    lib = _load()
    rp, ci = _i64(rp), _i32(ci)
    nnz = int(rp[-1])
    trp = np.zeros(n + 1, dtype=np.int64)
    tci = np.zeros(max(nnz, 1), dtype=np.int32)
    tv = np.zeros(max(nnz, 1), dtype=np.float64)
    vv = _f64(v) if v is not None else None
    lib.orc_transpose(n, _p(rp), _p(ci), _p(vv) if vv is not None else None, _p(trp), _p(tci),
                      _p(tv) if vv is not None else None)
    return trp, tci[:nnz].copy(), (tv[:nnz].copy() if v is not None else None)


def apply_t(n, trp, tci, tv, p):
    """y = (L~U~)^-T p on the transposed factors (U~^T then L~^T sweeps)."""
    return _vec_call("orc_apply_t", n, trp, tci, tv, p)


def iiluk_build(n, frp, fci, fv):
    """TPIILU incomplete inverses (Sec. 3.5), aligned with F's pattern."""
    lib = _load()
    frp, fci, fv = _i64(frp), _i32(fci), _f64(fv)
    g = np.zeros(max(int(frp[-1]), 1), dtype=np.float64)
    lib.orc_iiluk_build(n, _p(frp), _p(fci), _p(fv), _p(g))
    return g[: int(frp[-1])].copy()


def iiluk_apply(n, frp, fci, g, p):
    """y = (I + G_U) D^-1 (I + G_L) p (Eq. forwardsubB and its mirror)."""
    return _vec_call("orc_iiluk_apply", n, frp, fci, g, p)


def dot(x, y, mode=DOT_SEQ):
    lib = _load()
    x, y = _f64(x), _f64(y)
    return lib.orc_dot(len(x), _p(x), _p(y), mode)


def spmv(n, rp, ci, v, x):
    return _vec_call("orc_spmv", n, rp, ci, v, x)


def gmres(n, arp, aci, av, b, prec_kind=PREC_NONE, F=None, restart=30, rtol=1e-8, maxit=10000,
          dotmode=DOT_SEQ, prec_transpose=False, update=UPDATE_Z):
    """Right-preconditioned restarted GMRES(m), x0 = 0.

    ``F`` is (rowptr, colind, values) of the factors (ILU), their transpose
    (ILU with prec_transpose), or the TPIILU array g (IILU).  ``update``:
    UPDATE_Z ends a cycle with x += Z y on the kept preconditioned basis (the
    flexible form); UPDATE_MVY with x += M^-1 (V y) (the textbook form of
    right preconditioning, Sec. 2's A U~^-1 L~^-1).
    Returns (status, x, iterations, relres, cycles)."""
    lib = _load()
    arp, aci, av, b = _i64(arp), _i32(aci), _f64(av), _f64(b)
    x = np.zeros(max(n, 1), dtype=np.float64)
    info = np.zeros(3, dtype=np.float64)
    if F is None:
        frp = fci = fv = None
    else:
        frp, fci, fv = _i64(F[0]), _i32(F[1]), _f64(F[2])
    st = lib.orc_gmres_update(n, _p(arp), _p(aci), _p(av), prec_kind, int(prec_transpose),
                              _p(frp) if frp is not None else None,
                              _p(fci) if fci is not None else None,
                              _p(fv) if fv is not None else None, _p(b), _p(x), restart, rtol,
                              maxit, dotmode, int(update), _p(info))
    return st, x[:n].copy(), int(info[0]), float(info[1]), int(info[2])


def bicgstab(n, arp, aci, av, b, prec_kind=PREC_NONE, F=None, rtol=1e-8, maxit=10000,
             dotmode=DOT_SEQ):
    """Right-preconditioned BiCGSTAB, x0 = 0 (the iteration written out in
    iluk_oracle.c).  ``F`` as for gmres (no transpose).
    Returns (status, x, iterations, true relres, ended_at_half_step)."""
    lib = _load()
    arp, aci, av, b = _i64(arp), _i32(aci), _f64(av), _f64(b)
    x = np.zeros(max(n, 1), dtype=np.float64)
    info = np.zeros(3, dtype=np.float64)
    if F is None:
        frp = fci = fv = None
    else:
        frp, fci, fv = _i64(F[0]), _i32(F[1]), _f64(F[2])
    st = lib.orc_bicgstab(n, _p(arp), _p(aci), _p(av), prec_kind,
                          _p(frp) if frp is not None else None,
                          _p(fci) if fci is not None else None,
                          _p(fv) if fv is not None else None, _p(b), _p(x), rtol, maxit, dotmode,
                          _p(info))
    return st, x[:n].copy(), int(info[0]), float(info[1]), bool(info[2])


def tpilu(n, arp, aci, av, b, F, g, solver="gmres", restart=50, rtol=1e-8, iilu_maxit=50,
          maxit=10000, dotmode=DOT_SEQ):
    """The TPILU(k) solve policy of Sec. 1 composed from the solvers above:
    TPIILU first with at most ``iilu_maxit`` iterations, and if it does not
    converge (or breaks down), ILU(k) from x0 = 0.  ``F`` = (rowptr, colind,
    values) of the factors, ``g`` their TPIILU array.
    Returns (status, x, iterations, relres, used) with used "iilu" or "ilu"."""
    def run(kind, Fa, its):
        if solver == "gmres":
            st, x, it, rel, _ = gmres(n, arp, aci, av, b, kind, Fa, restart, rtol, its, dotmode)
        else:
            st, x, it, rel, _ = bicgstab(n, arp, aci, av, b, kind, Fa, rtol, its, dotmode)
        return st, x, it, rel
    st, x, it, rel = run(PREC_IILU, (F[0], F[1], g), iilu_maxit)
    if st == OK:
        return st, x, it, rel, "iilu"
    st, x, it, rel = run(PREC_ILU, F, maxit)
    return st, x, it, rel, "ilu"


def adjoint(n, arp, aci, av, frp, fci, fv, x, gx, restart=30, rtol=1e-8, maxit=10000,
            dotmode=DOT_SEQ):
    """A^T lambda = gx with (L~U~)^-T preconditioning; dL/da_ij = -lambda_i x_j.

    Returns (status, lambda, gA, iterations, relres)."""
    lib = _load()
    arp, aci, av = _i64(arp), _i32(aci), _f64(av)
    frp, fci, fv = _i64(frp), _i32(fci), _f64(fv)
    x, gx = _f64(x), _f64(gx)
    lam = np.zeros(max(n, 1), dtype=np.float64)
    gA = np.zeros(max(int(arp[-1]), 1), dtype=np.float64)
    info = np.zeros(3, dtype=np.float64)
    st = lib.orc_adjoint(n, _p(arp), _p(aci), _p(av), _p(frp), _p(fci), _p(fv), _p(x), _p(gx),
                         _p(lam), _p(gA), restart, rtol, maxit, dotmode, _p(info))
    return st, lam[:n].copy(), gA[: int(arp[-1])].copy(), int(info[0]), float(info[1])


def factor(A, k):
    """Convenience: symbolic + numeric on a workloads.CSR.  Returns a dict."""
    st, bad, frp, fci, flev = symbolic(A.n, A.rowptr, A.colind, k)
    if st != OK:
        raise OracleError(st, bad, "symbolic")
    st, bad, fv = numeric(A.n, A.rowptr, A.colind, A.val, frp, fci)
    if st != OK:
        raise OracleError(st, bad, "numeric")
    return {"rowptr": frp, "colind": fci, "level": flev, "val": fv}
