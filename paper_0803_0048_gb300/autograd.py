"""a8: differentiable solve x = A(theta)^-1 b with a hand-written adjoint.

Forward: ILU(k) numeric factorization of A's values on a fixed symbolic
pattern, then right-preconditioned GMRES(m).  Backward, for an incoming
gradient g = dL/dx: solve A^T lambda = g by GMRES on the explicit transpose of
A, preconditioned with the same factors transposed, (L~U~)^-T = L~^-T U~^-T
(a U~^T sweep then an L~^T sweep); then dL/db = lambda and
dL/da_ij = -lambda_i x_j on A's stored entries.  The assembly A(theta) is
ordinary torch code, so autograd carries dL/da on to theta.  Every numerical
step runs in libiluk's kernels.
"""
from __future__ import annotations

import torch

from . import api


class IlukSolver:
    """A fixed pattern and the solver settings; the symbolic phase runs once."""

    def __init__(self, rowptr: torch.Tensor, colind: torch.Tensor, k: int, restart: int = 30,
                 rtol: float = 1e-8, maxit: int = 10000, basis: str = "auto"):
        # basis: what each GMRES cycle (forward and adjoint) keeps for its
        # final update.  "store" keeps the m preconditioned basis vectors;
        # "recompute" keeps only the Krylov basis and applies the factors
        # again at the end of a cycle (same bits, m vectors less memory);
        # "auto" stores them when they fit in half of the free device memory.
        self.rowptr, self.colind = rowptr, colind
        self.k, self.restart, self.rtol, self.maxit = k, restart, rtol, maxit
        self.basis = basis
        self.S = api.symbolic(rowptr, colind, k)
        self.last_forward = None
        self.last_backward = None

    def solve(self, vals: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        return IlukSolve.apply(vals, b, self)


class IlukSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, solver: IlukSolver):
        vals_d = vals.detach().contiguous()
        b_d = b.detach().contiguous()
        F = api.numeric(solver.S, vals_d)
        x, info = api.gmres(solver.rowptr, solver.colind, vals_d, b_d, F, restart=solver.restart,
                            rtol=solver.rtol, maxit=solver.maxit, basis=solver.basis)
        solver.last_forward = info
        ctx.solver = solver
        ctx.F = F
        ctx.save_for_backward(vals_d, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        vals_d, x = ctx.saved_tensors
        s = ctx.solver
        lam, info = api.gmres(s.rowptr, s.colind, vals_d, gx.detach().contiguous(), ctx.F,
                              restart=s.restart, rtol=s.rtol, maxit=s.maxit, transpose=True,
                              basis=s.basis)
        s.last_backward = info
        gA = api.adjoint_scatter(s.rowptr, s.colind, lam, x)
        return gA, lam, None


def solve(vals: torch.Tensor, b: torch.Tensor, solver: IlukSolver) -> torch.Tensor:
    return IlukSolve.apply(vals, b, solver)
