"""Differentiable all-at-once heat solve: u = T(a)^{-1} f_H(f, u0[, u^(-1)]) as a torch autograd op.

Forward: st_assemble_rhs + st_solve (preconditioned MINRES on Y T u = Y f_H).
Backward: the blocks of T are symmetric, so T^T = Y T Y and the same preconditioned MINRES
solves T^T lam = dL/du (st_solve_transpose); st_grad_rhs maps lam to dL/df, dL/du0, dL/du^(-1)
and st_grad_a contracts lam with the solution into dL/da at the nodes.  Every step runs in the
library's kernels; this module only wires them into torch.autograd.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Optional

import torch

from . import ProblemSpec, Solver


class _HeatSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, u0, a_nodal, u_prev, spec: ProblemSpec, tol: float, maxit: int):
        a_host = None
        if a_nodal is not None:
            a_host = a_nodal.detach().to("cpu", torch.float64).contiguous().numpy()
        s = Solver(replace(spec, a_nodal=a_host))
        fH = s.st_assemble_rhs(f.detach().contiguous(), u0.detach().contiguous(),
                               None if u_prev is None else u_prev.detach().contiguous())
        u, stats = s.st_solve(fH, tol=tol, maxit=maxit)
        ctx.solver = s
        ctx.tol, ctx.maxit = tol, maxit
        ctx.has_a = a_nodal is not None
        ctx.a_shape = None if a_nodal is None else a_nodal.shape
        ctx.has_uprev = u_prev is not None
        ctx.stats = stats
        ctx.save_for_backward(u, u0)
        return u.view(spec.n, spec.m)

    @staticmethod
    def backward(ctx, gu):
        u, u0 = ctx.saved_tensors
        s = ctx.solver
        lam, _ = s.st_solve_transpose(gu.contiguous().view(-1), tol=ctx.tol, maxit=ctx.maxit)
        gf, gu0, gup = s.st_grad_rhs(lam)
        ga = None
        if ctx.has_a and ctx.needs_input_grad[2]:
            ga = s.st_grad_a(lam, u, u0.detach().contiguous()).view(ctx.a_shape)
        s.close()
        return (gf if ctx.needs_input_grad[0] else None,
                gu0 if ctx.needs_input_grad[1] else None,
                ga,
                gup if (ctx.has_uprev and ctx.needs_input_grad[3]) else None,
                None, None, None)


def heat_solve(f: torch.Tensor, u0: torch.Tensor, spec: ProblemSpec,
               a_nodal: Optional[torch.Tensor] = None, u_prev: Optional[torch.Tensor] = None,
               tol: float = 1e-10, maxit: int = 500) -> torch.Tensor:
    """Solve the all-at-once system; differentiable in f ((n+1) x m), u0 (m), the nodal a
    ((my+2) x (mx+2), or mx+2 in 1D; spec.a_nodal is ignored when given) and u^(-1) (BDF2).
    Returns u as an (n, m) CUDA float64 tensor."""
    return _HeatSolve.apply(f, u0, a_nodal, u_prev, spec, tol, maxit)
