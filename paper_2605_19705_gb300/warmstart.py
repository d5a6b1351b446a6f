"""Learned warm start x0 = A^T y + W_phi(A^T y): data generation and training.

The paper leaves the initial point x^0 of Algorithm 1 free.  Here a small ReLU
conv net W_phi is trained, with the library's own forward, reverse,
weight-gradient and Adam kernels (ideq_warm_train_step), to map the
back-projection A^T y to equilibria that the plain solver itself produces, and is
then used as IDEQ_INIT_WARM.  The plain solver from A^T y stays the fallback and
the judge of the warm start's error: both reach the same stopping residual.
This module only orchestrates calls into the C ABI.
"""
from __future__ import annotations

import torch

from . import binding as B


def equilibria(ctx, op, y, params):
    """(A^T y, x_bar) for a batch: the plain solve from x0 = A^T y."""
    aty = B.ideq_apply_AT(ctx, op, y)
    p = B.make_params(params.lam, params.tau, params.beta, params.restart_B or float("inf"),
                      params.tol, params.max_iter, B.IDEQ_INIT_ATY)
    x, _ = B.ideq_solve(ctx, op, y, p, allow_maxiter=True)
    return aty, x


def warm_set(ctx, desc, weights):
    import torch as _t
    ctx.check(B._lib.ideq_warm_set(ctx.h, B.ctypes.byref(desc), B._ptr(weights, _t.float32)))


def warm_forward(ctx, aty, out=None):
    out = torch.empty_like(aty) if out is None else out
    ctx.check(B._lib.ideq_warm_forward(ctx.h, B._shape(aty), B._ptr(aty, torch.float32),
                                       B._ptr(out, torch.float32)))
    return out


def warm_train_step(ctx, aty, target, lr, loss=None):
    """One Adam step on mean((aty + W(aty) - target)^2); loss (device double[1]) is
    filled with the loss before the step."""
    ctx.check(B._lib.ideq_warm_train_step(ctx.h, B._shape(aty), B._ptr(aty, torch.float32),
                                          B._ptr(target, torch.float32), float(lr),
                                          B._ptr(loss, torch.float64)))


def warm_get(ctx, nparams):
    w = torch.empty(nparams, dtype=torch.float32, device="cuda")
    ctx.check(B._lib.ideq_warm_get(ctx.h, B._ptr(w, torch.float32)))
    return w


def train(ctx, atys, targets, steps=300, lr=1e-3, batch=8, seed=0):
    """Adam training of the warm start on (A^T y, x_bar) pairs, minibatches drawn
    with a seeded generator; returns the per-step losses (host list)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = atys.shape[0]
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    hist = []
    for _ in range(steps):
        idx = torch.randperm(n, generator=g)[:batch].to(atys.device)
        a = atys.index_select(0, idx).contiguous()
        t = targets.index_select(0, idx).contiguous()
        warm_train_step(ctx, a, t, lr, loss)
        hist.append(loss)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    return [float(h.item()) for h in hist]
