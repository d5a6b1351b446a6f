"""torch.autograd.Function over the library's solve and implicit backward.

Forward: x_hat = ideq_solve(y; theta, lambda) (Algorithm 1).  Backward: the
gradients of the loss with respect to theta (the flat weight vector) and lambda
from ideq_solve_backward -- the implicit differentiation of the fixed point
(App. D.1.2), or its Jacobian-free estimate (JFB, App. D.1.1).  Marshalling only:
both directions run in the CUDA library.
"""
from __future__ import annotations

import torch

from . import binding as B


class IDEQSolve(torch.autograd.Function):
    """Implicit differentiation assumes x_hat is a fixed point and u solves the
    adjoint equation: a forward solve with a stopping tolerance that hits max_iter
    (IDEQ_MAXITER), a diverged image, or an implicit adjoint solve that hits its cap
    (IDEQ_ADJ_MAXITER) raises IdeqError instead of returning a gradient.  A fixed
    run (params.tol == 0) is a K-step map and ends at max_iter by definition."""

    @staticmethod
    def forward(fctx, weights, lam, y, ctx, op, params, adj):
        B.ideq_set_weights(ctx, weights.detach().contiguous())
        params.lam = float(lam)
        x, _ = B.ideq_solve(ctx, op, y, params, allow_maxiter=params.tol == 0.0)
        fctx.ictx, fctx.op, fctx.params, fctx.adj = ctx, op, params, adj
        fctx.save_for_backward(weights, y, x)
        return x

    @staticmethod
    def backward(fctx, gx):
        weights, y, x = fctx.saved_tensors
        dtheta = torch.empty_like(weights)
        dlam = torch.empty(1, dtype=torch.float32, device=weights.device)
        B.ideq_solve_backward(fctx.ictx, fctx.op, y, x, gx.contiguous().float(), fctx.params,
                              fctx.adj, dtheta, dlam, allow_maxiter=False)
        return dtheta, dlam.reshape(()), None, None, None, None, None


make_adj = B.make_adj


def ideq_restore(weights, lam, y, ctx, op, params, adj):
    """Differentiable restoration x_hat(theta, lambda)."""
    return IDEQSolve.apply(weights, lam, y, ctx, op, params, adj)
