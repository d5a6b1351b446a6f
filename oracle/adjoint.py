"""Implicit differentiation of the i-DEQ fixed point (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

At a fixed point xbar = T(xbar, xbar) of T(x1, x2) = R(x1 + beta (x1 - x2)),
R(z) = z - tau (grad f(z) + lambda grad g_theta(z)), implicit differentiation
(App. D.1.2) gives

    d xbar / d Theta = (I - dT/dx1 - dT/dx2)^{-1} dT/dTheta.

Here dT/dx1 + dT/dx2 = (1 + beta) J_R - beta J_R = J_R with
J_R = I - tau (H_f + lambda H_g) at xbar, a symmetric matrix, so the transposed
and untransposed forms of the paper coincide.  For a loss l with v = dl/dxbar the
parameter gradient is (dT/dTheta)^T u where u solves u = J_R^T u + v, and

    dT/dtheta  = -tau lambda d(grad g_theta(xbar))/dtheta
    dT/dlambda = -tau grad g(xbar)

(dT/dtau and dT/dalpha vanish at the exact fixed point, Remark after App. D.1.2).
JFB (Jacobian-free backpropagation, App. D.1.1) replaces u by v.
"""
from __future__ import annotations

import math

import numpy as np

from . import nets


def JR_T(net, op, y, xbar, u, lam, tau):
    """J_R^T u = u - tau (H_f u + lambda H_g u) at xbar."""
    return u - tau * (op.hvp_f(xbar, y, u) + lam * nets.hvp_g(net, xbar, u))


def adjoint_solve(net, op, y, xbar, v, lam, tau, tol=1e-3, max_iter=1000, beta=0.0):
    """Fixed-point iteration u <- J_R^T u + v (optionally heavy-ball with beta).

    Stops when ||u^{k+1} - u^k|| / ||u^k|| < tol.  Returns (u, iterations, converged)."""
    u = np.asarray(v, dtype=np.float64).copy()
    u_prev = u.copy()
    for it in range(1, max_iter + 1):
        w = u + beta * (u - u_prev)
        u_new = JR_T(net, op, y, xbar, w, lam, tau) + v
        s = float(np.linalg.norm(u_new - u))
        nu = float(np.linalg.norm(u))
        u_prev, u = u, u_new
        if not math.isfinite(s):
            return u, it, False
        if s < tol * nu:
            return u, it, True
    return u, max_iter, False


def backward_image(net, op, y, xbar, v, lam, tau, mode="implicit", tol=1e-3,
                   max_iter=1000, beta=0.0):
    """(dl/dtheta flat, dl/dlambda, info) for one image."""
    if mode == "jfb":
        u, it, ok = np.asarray(v, dtype=np.float64), 0, True
    else:
        u, it, ok = adjoint_solve(net, op, y, xbar, v, lam, tau, tol, max_iter, beta)
    gtheta = -tau * lam * nets.grad_theta_dot(net, xbar, u)
    gg, _ = nets.grad_g(net, xbar)
    glam = -tau * float(np.sum(u * gg))
    return gtheta, glam, {"adj_iters": it, "adj_converged": ok, "u": u}


def mse_loss_grad(xhat, x_true):
    """l = mean((xhat - x*)^2) over the whole batch; returns (l, dl/dxhat)."""
    d = np.asarray(xhat, np.float64) - np.asarray(x_true, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward_batch(net, ops, ys, xbars, vs, lam, tau, mode="implicit", tol=1e-3,
                   max_iter=1000, beta=0.0):
    gt = np.zeros(net.nparams)
    gl = 0.0
    infos = []
    for i in range(len(ops)):
        a, b, inf = backward_image(net, ops[i], ys[i], xbars[i], vs[i], lam, tau, mode, tol,
                                   max_iter, beta)
        gt += a
        gl += b
        infos.append(inf)
    return gt, gl, infos
