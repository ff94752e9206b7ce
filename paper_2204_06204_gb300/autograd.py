"""torch.autograd.Function for the compliance through a truncated lower-level solve.

forward:  J(rho) = f^T u_T, T constant-beta Jacobi steps from u_0 = 0
          (``to_compliance_truncated``; the library keeps the iterates, all of them
          or every s-th with ``to_params.adj_stride``)
backward: dJ/drho by the library's reverse sweep (``to_compliance_truncated_grad``)

A problem keeps the iterates of its most recent forward call only.  Each forward
records the library's identifier of the iterates it left; when backward finds a
different identifier (another forward on the same problem ran in between, or the
design changed), it re-runs its own forward from the saved rho first, so several
graphs may share one problem.  Both directions run in the CUDA library; this
module only passes tensors.
"""
from __future__ import annotations

import torch

from . import to_compliance_truncated, to_compliance_truncated_grad, to_compliance_truncated_id


class TruncatedCompliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, problem, T, beta):
        rho_c = rho.detach().contiguous()
        J = to_compliance_truncated(problem, rho_c, T, beta, want_J=True)
        ctx.problem, ctx.T, ctx.beta = problem, int(T), float(beta)
        ctx.fwd_id = to_compliance_truncated_id(problem)
        ctx.save_for_backward(rho_c)
        return torch.tensor(J, dtype=rho.dtype, device=rho.device)

    @staticmethod
    def backward(ctx, grad_out):
        P = ctx.problem
        (rho_c,) = ctx.saved_tensors
        if to_compliance_truncated_id(P) != ctx.fwd_id:
            to_compliance_truncated(P, rho_c, ctx.T, ctx.beta, want_J=False)
        g = P.elem()
        to_compliance_truncated_grad(P, float(grad_out.item()), g)
        return g, None, None, None


def compliance(rho, problem, T=5, beta=0.5):
    """J(rho) as a differentiable scalar (the problem must use the Jacobi preconditioner)."""
    return TruncatedCompliance.apply(rho, problem, T, beta)
