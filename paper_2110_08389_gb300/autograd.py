"""Differentiation through the multigrid solve (torch.autograd).

``tweed_solve(grid, f, g, **params)`` returns u, the solution of Eq. prob:DP
(Sec. 2) with source f at the interior nodes and Dirichlet data g on the
boundary nodes, solved by the library's multigrid (tweed smoothing by
default, FP64 or FP32 cycles with FP64 refinement).  It is differentiable in
f and g.  With A the interior operator and B the coupling of interior rows to
boundary values, u_int = A^{-1} (f - B g) and u_b = g_b, so for a loss l(u)

    dl/df = lambda,   A^T lambda = dl/du_int      (mg_solve_adjoint)
    dl/dg_b = dl/du_b - sum_p coef(p -> b) lambda_p   (mg_boundary_adjoint)

Both steps run in the CUDA library; this module only marshals tensors.
f, g: float64 CUDA tensors of shape (ny+1, nx+1); only the interior of f and
the boundary of g are used (their other entries get zero gradient).
"""
from __future__ import annotations

import torch

from . import mg


def _params(**kw) -> mg.Params:
    kw.setdefault("smoother", "tweed")
    kw.setdefault("tol", 1e-12)
    kw.setdefault("max_cycles", 200)
    kw.setdefault("max_outer", 40)
    kw["use_initial_guess"] = 0
    return mg.default_params(**kw)


class TweedSolve(torch.autograd.Function):
    """u = solve(f, g) with the adjoint multigrid solve as its backward."""

    @staticmethod
    def forward(ctx, f, g, grid: mg.Grid, params: mg.Params):
        for name, t in (("f", f), ("g", g)):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
                raise TypeError(f"{name}: contiguous float64 CUDA tensor expected")
        u = g.detach().clone()
        res = grid.solve(u, f.detach(), params)
        if res.status != mg.OK:
            raise mg.MGError(res.status, "mg_solve (forward)", f"relative residual {res.rel_res:.3e}")
        ctx.grid, ctx.params = grid, params
        return u

    @staticmethod
    def backward(ctx, grad_u):
        grid, params = ctx.grid, ctx.params
        gu = grad_u.detach().contiguous().to(torch.float64)
        lam = torch.zeros_like(gu)
        res = grid.solve_adjoint(lam, gu, params)
        if res.status != mg.OK:
            raise mg.MGError(res.status, "mg_solve_adjoint (backward)", f"relative residual {res.rel_res:.3e}")
        grad_g = torch.empty_like(gu)
        grid.boundary_adjoint(lam, gu, grad_g)
        return lam, grad_g, None, None


def tweed_solve(grid: mg.Grid, f: torch.Tensor, g: torch.Tensor, params: mg.Params | None = None, **kw):
    """Differentiable solve of Eq. prob:DP: u with u = g on the boundary and
    L u = f inside.  Keyword arguments are mg_params fields (smoother, nu1,
    nu2, cycle, restriction, precision, tol, ...)."""
    return TweedSolve.apply(f, g, grid, params or _params(**kw))
