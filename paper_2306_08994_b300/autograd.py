"""torch.autograd.Function over the C ABI: x = A(K)^-1 b with A = sum_e P_e^T K_e P_e.

Forward factors and solves (mf_factor + mf_solve, optionally refined).
Backward reuses the stored factors for the transposed solve
lambda = A^-T dL/dx (mf_solve_adjoint) and forms dL/dK_e = -lambda_e x_e^T
(mf_element_outer) and dL/db = lambda.  For a per-element parameter theta_e
with dK_e/dtheta_e given, mf_element_grad gives -lambda_e^T dK_e x_e directly.
"""
from __future__ import annotations

import torch

from .mfsolve import Factors


class MFSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values: torch.Tensor, b: torch.Tensor, factors: Factors, refine_tol: float = 0.0):
        values = values.contiguous()
        factors.factor(values)
        x = torch.empty_like(b)
        if refine_tol > 0:
            factors.refine_solve(values, b.contiguous(), x, tol=refine_tol, maxit=20)
        else:
            x.copy_(b)
            factors.solve(x)
        ctx.factors = factors
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        (x,) = ctx.saved_tensors
        f: Factors = ctx.factors
        lam = gx.contiguous().clone()
        f.solve(lam, adjoint=True)
        gK = None
        if ctx.needs_input_grad[0]:
            gK = torch.empty(f.analysis.n_elem * f.analysis.npe * f.analysis.npe, dtype=torch.float64,
                             device=x.device)
            f.element_outer(lam, x, gK)
        gb = lam if ctx.needs_input_grad[1] else None
        return gK, gb, None, None
