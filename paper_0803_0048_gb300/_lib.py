"""ctypes loader for libiluk.so and the C structs of include/iluk.h.

Argument marshalling only: every computation happens in the CUDA library.
If the library has not been built, loading fails with an error (there is no
fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libiluk.so")

OK, EINVAL, EPATTERN, ENODIAG, EZEROPIVOT, ENONFINITE, ENOMEM, ETIMEOUT, ENOCONV, ECUDA = range(10)
PREC_NONE, PREC_ILU, PREC_IILU = 0, 1, 2
# what a GMRES cycle keeps for its final update (gmres_solve_ex)
BASIS = {"auto": 0, "store": 1, "recompute": 2, "minv_vy": 3}
SOLVER_GMRES, SOLVER_BICGSTAB = 0, 1
SCHED_AUTO, SCHED_FLAGS, SCHED_SINGLE_CTA, SCHED_CLUSTER, SCHED_WARP_GRID, SCHED_WARP_CLUSTER = 0, 1, 2, 3, 4, 5
SCHED_WARP_CLUSTER_HELP = 6
_SCHED_NAMES = ["auto", "lockstep_grid", "lockstep_cta", "lockstep_cluster", "warp_grid",
                "warp_cluster", "warp_cluster_help"]


def sched_width(kind: int, threads: int) -> int:
    """Schedule byte of a warp-per-row kind at `threads` per CTA (ILUK_SCHED_WIDTH)."""
    return kind | ((threads // 128) << 4)


def sched_name(byte: int) -> str:
    """Readable name of one schedule byte, e.g. 'warp_cluster/512'."""
    kind, w = byte & 0xF, (byte >> 4) & 0xF
    name = _SCHED_NAMES[kind] if kind < len(_SCHED_NAMES) else f"kind{kind}"
    return f"{name}/{w * 128}" if w else name
PROF_KINDS = ["validate", "symbolic", "compact", "depth", "numeric", "sweep", "transpose",
              "iilu_build", "iilu_apply", "spmv", "dot", "vector", "sweep_bwd", "batch",
              "overlapped", "factor"]


class Pattern(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("colind", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("row", C.c_int64),
                ("relres", C.c_double), ("need", C.c_int64), ("cycles", C.c_int32),
                ("reserved", C.c_int32)]


class BatchItem(C.Structure):
    _fields_ = [("S", C.c_void_p), ("a_rowptr", C.c_void_p), ("a_colind", C.c_void_p),
                ("a_val", C.c_void_p), ("b", C.c_void_p), ("x", C.c_void_p)]


class SymView(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("colind", C.c_void_p), ("level", C.c_void_p), ("diag", C.c_void_p),
                ("a2f", C.c_void_p), ("max_row", C.c_int32), ("depth_lower", C.c_int32),
                ("depth_upper", C.c_int32), ("k", C.c_int32)]


# (name, restype, argtypes) for every entry point declared in include/iluk.h
P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
PP = C.POINTER(C.c_void_p)
SIGNATURES = [
    ("iluk_strerror", C.c_char_p, [I]),
    ("iluk_set_wait_limit", I64, [I64]),
    ("iluk_debug_hold_row", I64, [I64]),
    ("iluk_set_symbolic_variant", I, [I]),
    ("iluk_launch_count", I64, []),
    ("iluk_prof_enable", I, [I]),
    ("iluk_prof_read", I, [P, P, I]),
    ("iluk_validate", I, [P, P, P]),
    ("iluk_symbolic", I, [P, I, PP, P, P]),
    ("iluk_sym_query", I, [P, P]),
    ("iluk_sym_depth", I, [P, P, P, P]),
    ("iluk_sym_export", I, [P, P, P, P, P, P]),
    ("iluk_sym_destroy", None, [P]),
    ("iluk_numeric", I, [P, P, PP, P, P]),
    ("iluk_refactor", I, [P, P, P, P]),
    ("iluk_factor", I, [P, P, I, PP, PP, P, P]),
    ("iluk_fac_values", I, [P, PP]),
    ("iluk_fac_export", I, [P, P, P]),
    ("iluk_fac_status", I, [P, P, P]),
    ("iluk_fac_destroy", None, [P]),
    ("iluk_apply", I, [P, P, P, I, P]),
    ("iluk_apply_sched", I, [P, P, P, I, I, P]),
    ("iluk_set_schedule", I, [P, I]),
    ("iluk_get_schedule", I, [P]),
    ("iiluk_build", I, [P, PP, P, P]),
    ("iiluk_values", I, [P, PP]),
    ("iiluk_export", I, [P, P, P]),
    ("iiluk_apply", I, [P, P, P, P]),
    ("iiluk_apply_noalloc", I, [I64, P, P, P, P, P, P, P]),
    ("iiluk_destroy", None, [P]),
    ("iluk_spmv", I, [P, P, P, P, P]),
    ("iluk_dot", I, [I64, P, P, P, P]),
    ("iluk_div_rn", I, [I64, P, P, P, P]),
    ("gmres_solve", I, [P, P, I, P, P, P, I, D, I, I, P, P]),
    ("gmres_solve_ex", I, [P, P, I, P, P, P, I, D, I, I, I, P, P]),
    ("iluk_transpose", I, [P, P, P, P, P, P]),
    ("iluk_solve", I, [P, P, I, P, P, I, D, I, I, P, P, P, P]),
    ("iluk_solve_host", I, [I64, I64, P, P, P, P, P, I, I, D, I, I, P, P]),
    ("bicgstab_solve", I, [P, P, I, P, P, P, D, I, P, P]),
    ("tpilu_solve", I, [P, P, P, P, I, P, P, I, D, I, I, P, P, P]),
    ("iluk_adjoint_scatter", I, [P, P, P, P, P]),
    ("iluk_numeric_batched", I, [P, I64, P, P, P, P]),
    ("iluk_batch_create", I, [P, I64, I, D, I, PP, P]),
    ("iluk_batch_solve", I, [P, P]),
    ("iluk_batch_results", I, [P, P, P]),
    ("iluk_batch_width", I, [P]),
    ("iluk_batch_spin", I, [P]),
    ("iluk_batch_set_schedule", I, [P, I, I]),
    ("iluk_batch_destroy", None, [P]),
]

_lock = threading.Lock()
_lib = None


def load() -> C.CDLL:
    """Load libiluk.so; raises if it was not built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"libiluk.so not found at {LIB_PATH}; build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    return [s[0] for s in SIGNATURES]
