"""ILU(k) preconditioning for sparse non-symmetric Ax = b on one GB300.

After Dong & Cooperman, "A Bit-Compatible Shared Memory Parallelization for
ILU(k) Preconditioning and a Bit-Compatible Generalization to Distributed
Memory" (arXiv 0803.0048).  The work runs in libiluk.so (CUDA, sm_103a,
declared in include/iluk.h); this package is its thin Python binding.
"""
from . import _lib
from .api import (BatchSolve, CsrPattern, Factors, IlukError, IncompleteInverse, Symbolic,
                  adjoint_scatter, bicgstab, debug_hold_row, div_rn, dot, factor, gmres,
                  iiluk_build, launch_count, numeric, numeric_batched, prof_enable, prof_read,
                  set_symbolic_variant, set_wait_limit, solve, solve_host, spmv, symbolic,
                  tpilu_solve, transpose, validate)
from .autograd import IlukSolve, IlukSolver

__all__ = ["BatchSolve", "CsrPattern", "Factors", "IlukError", "IlukSolve", "IlukSolver",
           "IncompleteInverse", "Symbolic", "adjoint_scatter", "bicgstab", "debug_hold_row",
           "div_rn", "dot", "factor", "gmres", "iiluk_build", "launch_count", "numeric",
           "numeric_batched", "prof_enable", "prof_read", "set_symbolic_variant",
           "set_wait_limit", "solve", "solve_host", "spmv", "symbolic", "tpilu_solve",
           "transpose", "validate"]
