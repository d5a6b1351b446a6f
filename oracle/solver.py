"""The i-DEQ inertial fixed-point iteration (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

One image at a time, following Algorithm 1 (forward pass) in the paper's order:

    z^k     = x^k + (1 - alpha)(x^k - x^{k-1})              inertial step, Eq. Momentum
    x^{k+1} = z^k - tau (grad f(z^k, y) + lambda grad g(z^k))   RED step at z, Eq. ideq
    k      <- k + 1
    if k sum_{i<k} ||x^{i+1} - x^i||^2 > B^2:  x^{-1}, x^0 <- x^k, k <- 0   (Eq. restart)

with beta = 1 - alpha.  Readings where the paper is silent or loose:
  * the restart resets the accumulated sum with k (Alg. 1); a separate total
    counter counts every update and is what max_iter bounds;
  * stopping (App. D.1.3): ||x^{k+1} - x^k|| / ||x^k|| < tol after an update;
    the image is then frozen at x^{k+1}; tol = 0 runs exactly max_iter updates;
  * the output is the last iterate, x_hat = x^K (Remark 1 allows dropping the
    averaging step); with average=True it is the averaging step of Algorithm 1,
    x_hat = (1 / (K0 + 1)) sum_{k=0}^{K0} z^k with K0 the first minimiser of
    ||x^{k+1} - x^k|| over floor(K/2) < k < K - 1, for a run of exactly K =
    max_iter updates without restarts (tol = 0, B = inf), K >= 5;
  * a non-finite step norm marks the image diverged and freezes it.
With prox=True the update is the proximal step of Algorithm 2 (i-DEQ-P):
x^{k+1} = prox_{tau f}(z^k - tau lambda grad g(z^k)) (Eq. red_prox with the inertial
step), with the restart of Algorithm 1 (the reading shared by both variants).
Alpha = 1 (beta = 0) is RED, i.e. gradient descent on F = f + lambda g (Sec. 2.1).
"""
from __future__ import annotations

import math

import numpy as np

from . import nets

RUNNING, CONVERGED, MAXITER, DIVERGED = 0, 1, 2, 3


def red_step(net, op, y, z, lam, tau, prox=False):
    """T^RED(z) = z - tau (grad f(z) + lambda grad g(z)), or with prox=True the
    proximal step T^RED-P(z) = prox_{tau f}(z - tau lambda grad g(z)) (Eq. red_prox);
    also f(z), g(z)."""
    gg, gval = nets.grad_g(net, z)
    fval = op.f(z, y)
    if prox:
        return op.prox_f(z - tau * lam * gg, y, tau), fval, gval
    gf = op.grad_f(z, y)
    return z - tau * (gf + lam * gg), fval, gval


def averaging_step(zs, steps):
    """Averaging step of Algorithm 1 for a run of K = len(steps) updates:
    K0 = argmin_{floor(K/2) < k < K-1} ||x^{k+1} - x^k|| (first minimiser) and
    x_hat = (1 / (K0 + 1)) sum_{k=0}^{K0} z^k.  zs[k] = z^k, steps[k] = ||x^{k+1} - x^k||."""
    K = len(steps)
    window = range(K // 2 + 1, K - 1)
    if len(window) == 0:
        raise ValueError("the averaging window floor(K/2) < k < K-1 is empty (K < 5)")
    K0 = min(window, key=lambda k: steps[k])
    return np.mean(np.stack(zs[:K0 + 1]), axis=0), K0


def solve_image(net, op, y, x0, lam, tau, beta, B=math.inf, tol=0.0, max_iter=50,
                keep_history=False, average=False, prox=False, on_update=None):
    """Run the iteration on one image.  Returns (x_hat, info dict).

    on_update(total, x_new, rel), when given, is called after every update with
    the update count, the new iterate and its relative step (read-only hook for
    recording; it does not change the iteration)."""
    if average and (tol > 0.0 or B < math.inf):
        raise ValueError("the averaging step needs a fixed run: tol = 0 and no restart")
    x = np.asarray(x0, dtype=np.float64).copy()
    x_prev = x.copy()
    k, S, total, restarts = 0, 0.0, 0, 0
    status = MAXITER
    info = {"steps": [], "rel": [], "energy_hist": []}
    fval = gval = float("nan")
    rel = float("nan")
    zs, norms = [], []
    while total < max_iter:
        z = x + beta * (x - x_prev)
        x_new, fval, gval = red_step(net, op, y, z, lam, tau, prox)
        s = float(np.sum((x_new - x) ** 2))
        if average:
            zs.append(z)
            norms.append(math.sqrt(s))
        nx = float(np.sum(x * x))
        x_prev, x = x, x_new
        k += 1
        total += 1
        S += s
        rel = math.sqrt(s) / math.sqrt(nx) if nx > 0 else math.inf
        if on_update is not None:
            on_update(total, x, rel)
        if keep_history:
            info["steps"].append(math.sqrt(s))
            info["rel"].append(rel)
            info["energy_hist"].append(fval + lam * gval)
        if not math.isfinite(s):
            status = DIVERGED
            break
        if tol > 0.0 and math.sqrt(s) < tol * math.sqrt(nx):
            status = CONVERGED
            break
        if k * S > B * B:
            x_prev = x.copy()
            k, S = 0, 0.0
            restarts += 1
    info.update(iters=total, restarts=restarts, status=status, rel_res=rel,
                f=fval, g=gval, energy=fval + lam * gval, x_prev=x_prev)
    if average and status == MAXITER:
        x, info["K0"] = averaging_step(zs, norms)
        if keep_history:
            info["z_hist"], info["step_hist"] = zs, norms
    return x, info


def solve_batch(net, ops, ys, x0s, lam, tau, beta, B=math.inf, tol=0.0, max_iter=50,
                keep_history=False, average=False, prox=False):
    """Independent solves of a batch (images never interact)."""
    xs, infos = [], []
    for i in range(len(ops)):
        x, inf = solve_image(net, ops[i], ys[i], x0s[i], lam, tau, beta, B, tol, max_iter,
                             keep_history, average, prox)
        xs.append(x)
        infos.append(inf)
    return np.stack(xs), infos


def psnr(x, x_true) -> float:
    """10 log10(1 / MSE), peak 1, no clipping."""
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(x_true, np.float64)) ** 2))
    return 10.0 * math.log10(1.0 / mse) if mse > 0 else math.inf


def step_batch(net, ops, ys, x, x_prev, lam, tau, beta):
    """One inertial RED update for every image from (x^k, x^{k-1}); returns x^{k+1}."""
    out = []
    for i in range(len(ops)):
        z = x[i] + beta * (x[i] - x_prev[i])
        out.append(red_step(net, ops[i], ys[i], z, lam, tau)[0])
    return np.stack(out)
