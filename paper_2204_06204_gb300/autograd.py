"""torch.autograd.Function for the compliance through a truncated lower-level solve.

forward:  J(rho) = f^T u_T, T constant-beta Jacobi steps from u_0 = 0
          (``to_compliance_truncated``; the library keeps the iterates)
backward: dJ/drho by the library's reverse sweep (``to_compliance_truncated_grad``)

Both directions run in the CUDA library; this module only passes tensors.
"""
from __future__ import annotations

import torch

from . import to_compliance_truncated, to_compliance_truncated_grad


class TruncatedCompliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, problem, T, beta):
        J = to_compliance_truncated(problem, rho.contiguous(), T, beta, want_J=True)
        ctx.problem = problem
        return torch.tensor(J, dtype=rho.dtype, device=rho.device)

    @staticmethod
    def backward(ctx, grad_out):
        P = ctx.problem
        g = P.elem()
        to_compliance_truncated_grad(P, float(grad_out.item()), g)
        return g, None, None, None


def compliance(rho, problem, T=5, beta=0.5):
    """J(rho) as a differentiable scalar (the problem must use the Jacobi preconditioner)."""
    return TruncatedCompliance.apply(rho, problem, T, beta)
