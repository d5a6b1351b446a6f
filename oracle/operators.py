"""Forward models A, adjoints and the data-fidelity term (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The problem is y = A(x) + n with data term f(x, y) = 1/2 ||A(x) - y||^2 and
gradient grad f(x) = J_A(x)^T (A(x) - y) (Sec. 1, Eq. inv_prob; the linear cases
App. E: grad f = A^T (A x - y), inpainting A = M).  Operators act on one image
of shape (c, h, w); blur kernels and masks are shared by the c channels.

  blur    : A x = k * x, circular 2-D convolution, kernel centre (kh//2, kw//2)
  mask    : A x = M . x, M in {0,1}^(h,w)                    (App. E, inpainting)
  satblur : A x = tanh(s (k * x)) / tanh(s), a smooth saturation after the blur
  rician  : denoising under Rician noise (App. E): f(x, y) = sum x^2 / (2 s^2)
            - log I0(x y / s^2), grad f = x / s^2 - (y / s^2) I1/I0(x y / s^2), with
            SciPy's exponentially scaled Bessel functions i0e, i1e as the primitive
  mri     : A x = M . F x for a complex image x stored as (re, im) channels, F the
            orthonormal 2-D DFT, M in {0,1}^(h,w) a k-space mask (App. E, MRI);
            A^T r = F^{-1}(M . r), prox_{tau f}(v) = F^{-1}((tau M y + F v) / (tau M + 1))
"""
from __future__ import annotations

import numpy as np


def conv_circ(x: np.ndarray, k: np.ndarray) -> np.ndarray:
    """(k * x)[i,j] = sum_{u,v} k[u,v] x[(i-(u-cy)) mod h, (j-(v-cx)) mod w]."""
    kh, kw = k.shape
    cy, cx = kh // 2, kw // 2
    out = np.zeros_like(x, dtype=np.float64)
    for u in range(kh):
        for v in range(kw):
            if k[u, v] != 0.0:
                out += float(k[u, v]) * np.roll(x, shift=(u - cy, v - cx), axis=(-2, -1))
    return out


def corr_circ(r: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Adjoint of conv_circ: sum_{u,v} k[u,v] r[(i+(u-cy)) mod h, (j+(v-cx)) mod w]."""
    kh, kw = k.shape
    cy, cx = kh // 2, kw // 2
    out = np.zeros_like(r, dtype=np.float64)
    for u in range(kh):
        for v in range(kw):
            if k[u, v] != 0.0:
                out += float(k[u, v]) * np.roll(r, shift=(-(u - cy), -(v - cx)), axis=(-2, -1))
    return out


def _cplx(x):
    return x[0] + 1j * x[1]


def _planes(z):
    return np.stack([z.real, z.imag])


class Operator:
    """Forward model of one image: kind in {"blur", "mask", "satblur", "mri"}."""

    def __init__(self, kind, kern=None, mask=None, gain=2.0, sigma=None):
        self.kind = kind
        self.sigma = None if sigma is None else float(sigma)
        if kind == "rician" and not (self.sigma and self.sigma > 0):
            raise ValueError("Rician operator needs sigma > 0")
        self.k = None if kern is None else np.asarray(kern, dtype=np.float64)
        self.m = None if mask is None else np.asarray(mask, dtype=np.float64)
        self.s = float(gain)
        if kind in ("blur", "satblur") and self.k is None:
            raise ValueError("blur operators need a kernel")
        if kind in ("mask", "mri") and self.m is None:
            raise ValueError("mask and MRI operators need a mask")

    @property
    def linear(self) -> bool:
        return self.kind != "satblur"

    def A(self, x):
        if self.kind == "rician":
            return np.asarray(x, np.float64)
        if self.kind == "blur":
            return conv_circ(x, self.k)
        if self.kind == "mask":
            return self.m * x
        if self.kind == "mri":
            return _planes(self.m * np.fft.fft2(_cplx(x), norm="ortho"))
        q = conv_circ(x, self.k)
        return np.tanh(self.s * q) / np.tanh(self.s)

    def AT(self, r):
        """Adjoint of the linear part: A^T for blur/mask, k^T (.) for satblur.

        For the saturation model this is the initialisation x0 = A^T y (the
        paper leaves x0 free, Alg. 1), not a Jacobian transpose."""
        if self.kind == "mask":
            return self.m * r
        if self.kind == "rician":
            return np.asarray(r, np.float64)
        if self.kind == "mri":
            return _planes(np.fft.ifft2(self.m * _cplx(r), norm="ortho"))
        return corr_circ(r, self.k)

    def JA(self, x, w):
        """Jacobian-vector product J_A(x) w."""
        if self.kind != "satblur":
            return self.A(w)
        q = conv_circ(x, self.k)
        sech2 = 1.0 - np.tanh(self.s * q) ** 2
        return (self.s / np.tanh(self.s)) * sech2 * conv_circ(w, self.k)

    def JAT(self, x, r):
        """Vector-Jacobian product J_A(x)^T r."""
        if self.kind != "satblur":
            return self.AT(r)
        q = conv_circ(x, self.k)
        sech2 = 1.0 - np.tanh(self.s * q) ** 2
        return corr_circ((self.s / np.tanh(self.s)) * sech2 * r, self.k)

    # data term -------------------------------------------------------------
    def f(self, x, y) -> float:
        if self.kind == "rician":  # log I0(t) = |t| + log i0e(t)
            from scipy.special import i0e
            s2 = self.sigma ** 2
            t = x * y / s2
            return float(np.sum(x * x / (2 * s2) - (np.abs(t) + np.log(i0e(t)))))
        e = self.A(x) - y
        return 0.5 * float(np.sum(e * e))

    def grad_f(self, x, y):
        if self.kind == "rician":  # I1/I0 = i1e/i0e
            from scipy.special import i0e, i1e
            s2 = self.sigma ** 2
            t = x * y / s2
            return x / s2 - (y / s2) * (i1e(t) / i0e(t))
        return self.JAT(x, self.A(x) - y)

    def prox_f(self, v, y, tau):
        """prox_{tau f}(v) = argmin_x 1/2||A x - y||^2 + 1/(2 tau)||x - v||^2 for the
        inpainting mask (App. E): (tau M y + v) / (tau M + 1) per pixel, i.e. v where
        the pixel is unobserved.  Other forward models have no closed form here."""
        if self.kind == "mri":  # k-space: (tau M y + F v) / (tau M + 1), App. E
            Y = (tau * self.m * _cplx(y) + np.fft.fft2(_cplx(v), norm="ortho")) / (tau * self.m + 1.0)
            return _planes(np.fft.ifft2(Y, norm="ortho"))
        if self.kind != "mask":
            raise NotImplementedError("closed-form prox only for the mask and MRI models")
        return (tau * self.m * y + v) / (tau * self.m + 1.0)

    def hvp_f(self, x, y, u):
        """Hessian of f at x applied to u.

        J_A^T J_A u + sum_i (A(x)-y)_i Hess(A_i) u; the second term vanishes for
        linear A.  For satblur, Hess(A_i) = (s/t)(-2 s tanh(s q_i) sech^2(s q_i))
        grad q_i grad q_i^T with q = k * x and t = tanh s."""
        if self.kind == "rician":  # (1/s^2 - (y/s^2)^2 B'(t)) u, B' = 1 - B/t - B^2
            from scipy.special import i0e, i1e
            s2 = self.sigma ** 2
            t = x * y / s2
            B = i1e(t) / i0e(t)
            with np.errstate(divide="ignore", invalid="ignore"):
                Bp = np.where(np.abs(t) > 1e-8, 1.0 - B / t - B * B, 0.5)
            return (1.0 / s2 - (y / s2) ** 2 * Bp) * u
        out = self.JAT(x, self.JA(x, u))
        if self.kind == "satblur":
            q = conv_circ(x, self.k)
            th = np.tanh(self.s * q)
            e = self.A(x) - y
            c2 = (self.s / np.tanh(self.s)) * (-2.0 * self.s) * th * (1.0 - th * th)
            out = out + corr_circ(e * c2 * conv_circ(u, self.k), self.k)
        return out

    def lipschitz_f(self) -> float:
        """Upper bound of the Lipschitz constant of grad f (linear: ||A||^2).

        Blur: max |K^|^2 over the DFT of the kernel on a 256-periodic grid bound
        by (sum |k|)^2; mask: 1 (App. E); satblur: (s / tanh s)^2 (sum|k|)^2
        plus the curvature term bounded the same way."""
        if self.kind == "mask":
            return 1.0
        l1 = float(np.abs(self.k).sum())
        if self.kind == "blur":
            return l1 * l1
        g = self.s / np.tanh(self.s)
        return g * g * l1 * l1 + 2.0 * g * self.s * l1 * l1


def make_operators(cfg: dict, wl: dict):
    """Per-image Operator list for a config and its drawn workload."""
    ops = []
    for i in range(cfg["n"]):
        kern = None if wl["kern"] is None else wl["kern"][i]
        mask = None if wl["mask"] is None else wl["mask"][i]
        sigma = cfg["noise_sigma"] if cfg["op"] == "rician" else None
        ops.append(Operator(cfg["op"], kern, mask, cfg.get("sat_gain", 2.0), sigma))
    return ops


def observe(ops, x_true, noise, mask=None):
    """y = A(x*) + n per image (FP64).  For inpainting y = M (x* + n); for MRI
    y = M (F x* + n), the noise (re, im planes) on the sampled k-space entries."""
    ys = []
    for i, op in enumerate(ops):
        if op.kind == "mask":
            ys.append(op.m * (x_true[i].astype(np.float64) + noise[i]))
        elif op.kind == "mri":
            ys.append(op.A(x_true[i].astype(np.float64)) + op.m * noise[i])
        elif op.kind == "rician":  # magnitude of x + n_re + i n_im (App. E)
            x = x_true[i].astype(np.float64)
            ys.append(np.sqrt((x + noise[i][0]) ** 2 + noise[i][1] ** 2))
        else:
            ys.append(op.A(x_true[i].astype(np.float64)) + noise[i])
    return np.stack(ys)
