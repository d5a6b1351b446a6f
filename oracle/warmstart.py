"""Learned warm start x0 = A^T y + W_phi(A^T y) (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper leaves the initial point free (Alg. 1: x^{-1} = x^0 in R^d).  The warm
start is a small 3x3 ReLU conv net W_phi applied in residual form to the
back-projection A^T y, trained with the mean squared error to equilibria of the
plain solver and updated with Adam (the optimiser the paper uses, App. D.1.3,
PyTorch defaults: beta1 = 0.9, beta2 = 0.999, eps = 1e-8).
"""
from __future__ import annotations

import numpy as np

from . import nets


def warm_forward(wnet, aty):
    """x0 = A^T y + W(A^T y) for one image."""
    out, _ = nets.forward(wnet, aty)
    return aty + out


def warm_loss_grad(wnet, atys, targets):
    """MSE over the batch of x0 against targets; returns (loss, flat grad)."""
    n_el = atys.size
    loss = 0.0
    grad = np.zeros(wnet.nparams)
    for i in range(atys.shape[0]):
        out, vals = nets.forward(wnet, atys[i])
        d = atys[i] + out - targets[i]
        loss += float(np.sum(d * d))
        _, gW = nets.vjp(wnet, vals, 2.0 * d / n_el, want_w=True)
        grad += wnet.flatten(gW)
    return loss / n_el, grad


class Adam:
    """Adam with bias correction (Kingma & Ba), PyTorch's default constants."""

    def __init__(self, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, p, g):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        return p - self.lr * mh / (np.sqrt(vh) + self.eps)
