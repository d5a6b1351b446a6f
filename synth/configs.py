"""Workload definitions C0-C4 and the seeded sampler that materialises them.

Each config fixes the shapes, the degradation, the regulariser network, the
solver parameters (lambda, tau, beta = 1 - alpha, restart bound B, stopping
tolerance, iteration cap) and the seeds.  ``workload`` draws every random input;
it applies no operator: y = A(x*) + n is formed by whichever side consumes it.

Solver-parameter readings (the paper tunes lambda, tau, alpha, B for pretrained
networks, Table 3; these networks are random):
  * beta = 1 - alpha = 0.8 (alpha = 0.2 in every row of Table 3), 0.5 for C0;
  * lambda = 0.1 (the "arb.init." value of Table 3);
  * tau below 1/(L_f + lambda L_g) with L_g estimated by power iteration on the
    Hessian of g (oracle.nets.estimate_lipschitz);
  * B = inf (no restart) for the headline runs, as in the paper's training and
    inference protocol (App. D.1.3); finite-B cases are separate test inputs;
  * stopping on ||x^{k+1}-x^k|| / ||x^k|| < tol (App. D.1.3, eps = 1e-4).
"""
from __future__ import annotations

import copy
import math

import numpy as np

from . import generators as G

INF = math.inf

UNET_FULL = {"type": "unet", "widths": [64, 128, 256, 512], "n_rb": 2, "act": "softplus"}
UNET_HALF = {"type": "unet", "widths": [32, 64, 128, 256], "n_rb": 2, "act": "softplus"}

CONFIGS = {
    # Plain method, tiny: 64x64 grey, 9x9 Gaussian blur sigma 1.6, fixed 50 steps.
    "C0": dict(n=1, c=1, h=64, w=64, op="blur",
               kernel={"type": "gauss", "size": 9, "sigma": 1.6},
               noise_sigma=0.01,
               net={"type": "cnn", "chans": [1, 32, 32, 32, 1], "act": "softplus"},
               lam=0.1, tau=0.8, beta=0.5, B=INF, tol=0.0, max_iter=50,
               precision="fp32",
               seeds={"img": 0, "noise": 1000, "weights": 2000, "kernel": 0, "mask": 0}),
    # Plain method at scale, motion blur: 8 x RGB 256^2, 25x25 random-walk kernels.
    "C1a": dict(n=8, c=3, h=256, w=256, op="blur",
                kernel={"type": "motion", "size": 25},
                noise_sigma=0.02, net=UNET_FULL,
                lam=0.1, tau=0.75, beta=0.8, B=INF, tol=1e-4, max_iter=3000,
                precision="fp32",
                seeds={"img": 0, "noise": 1000, "weights": 2001, "kernel": 3000, "mask": 0}),
    # Plain method at scale, inpainting keeping 30% of pixels.
    "C1b": dict(n=8, c=3, h=256, w=256, op="mask",
                kernel=None, mask_keep=0.30,
                noise_sigma=0.02, net=UNET_FULL,
                lam=0.1, tau=0.75, beta=0.8, B=INF, tol=1e-4, max_iter=3000,
                precision="fp32",
                seeds={"img": 0, "noise": 1000, "weights": 2001, "kernel": 0, "mask": 4000}),
    # Differentiation: 16 x RGB 128^2, per-image Gaussian sigma U[0.5,3], noise U[.005,.05].
    "C3": dict(n=16, c=3, h=128, w=128, op="blur",
               kernel={"type": "gauss_range", "size": 9, "sigma": [0.5, 3.0]},
               noise_sigma=[0.005, 0.05], net=UNET_HALF,
               lam=0.1, tau=0.75, beta=0.8, B=INF, tol=1e-3, max_iter=3000,
               adj_tol=1e-3, precision="fp32",
               seeds={"img": 5000, "noise": 5100, "weights": 2003, "kernel": 5200, "mask": 0}),
    # Warm start + saturation: A(x) = tanh(2 k*x)/tanh 2, 15x15 Gaussian sigma 2.
    "C4": dict(n=32, c=3, h=256, w=256, op="satblur", sat_gain=2.0,
               kernel={"type": "gauss", "size": 15, "sigma": 2.0},
               noise_sigma=0.01, net=UNET_FULL,
               warm={"type": "cnn", "chans": [3, 48, 48, 48, 48, 48, 3], "act": "relu"},
               lam=0.1, tau=0.2, beta=0.8, B=INF, tol=1e-4, max_iter=3000,
               precision="fp32",
               seeds={"img": 6000, "noise": 7000, "weights": 2001, "kernel": 0, "mask": 0,
                      "warm": 2004}),
    # MRI (App. E): 4 complex 256^2 images as (re, im) channels, Cartesian column
    # undersampling x4 with an 8% fully sampled centre, complex k-space noise on the
    # sampled entries; y = M (F x + n), F the orthonormal 2-D DFT.
    "C5": dict(n=4, c=2, h=256, w=256, op="mri",
               kernel=None, accel=4, center=0.08,
               noise_sigma=0.01, net=UNET_HALF,
               lam=0.1, tau=0.75, beta=0.8, B=INF, tol=1e-4, max_iter=3000,
               precision="fp32",
               seeds={"img": 8000, "noise": 8100, "weights": 2005, "kernel": 0, "mask": 8200}),
    # Rician denoising (App. E): 4 grey 256^2 images, y = |x + n_re + i n_im| with
    # sigma 25.5/255; L_f = 1/sigma^2, so tau ~ 0.9 sigma^2.
    "C6": dict(n=4, c=1, h=256, w=256, op="rician", kernel=None,
               noise_sigma=0.1, net=UNET_HALF,
               lam=0.1, tau=0.009, beta=0.8, B=INF, tol=1e-4, max_iter=3000,
               precision="fp32",
               seeds={"img": 8500, "noise": 8600, "weights": 2006, "kernel": 0, "mask": 0}),
}
CONFIGS["C2"] = dict(copy.deepcopy(CONFIGS["C1a"]), precision="bf16")


def get_config(name: str, **overrides) -> dict:
    cfg = copy.deepcopy(CONFIGS[name])
    cfg["name"] = name
    for k, v in overrides.items():
        cfg[k] = v
    return cfg


def net_layout(net: dict, c: int):
    if net["type"] == "unet":
        return G.unet_layout(c, net["widths"], net.get("n_rb", 2))
    return G.cnn_layout(net["chans"])


def workload(cfg: dict) -> dict:
    """Draw every seeded input of ``cfg``.

    Returns x_true (n,c,h,w) f32, kern (n,kh,kw) f32 or None, mask (n,h,w) u8 or
    None, noise (n,c,h,w) f32, weights (flat f32), and warm_weights when the
    config has a warm-start network.
    """
    n, c, h, w = cfg["n"], cfg["c"], cfg["h"], cfg["w"]
    s = cfg["seeds"]
    if cfg["op"] == "mri":
        x_true = np.stack([G.complex_image(s["img"] + i, h, w) for i in range(n)])
    else:
        x_true = G.synth_batch(s["img"], n, c, h, w)
    kern = None
    ks = cfg.get("kernel")
    if ks is not None:
        if ks["type"] == "gauss":
            k1 = G.gaussian_kernel(ks["size"], ks["sigma"])
            kern = np.stack([k1] * n)
        elif ks["type"] == "gauss_range":
            rng = np.random.default_rng(s["kernel"])
            sig = rng.uniform(ks["sigma"][0], ks["sigma"][1], n)
            kern = np.stack([G.gaussian_kernel(ks["size"], float(v)) for v in sig])
        elif ks["type"] == "motion":
            kern = np.stack([G.motion_kernel(s["kernel"] + i, ks["size"]) for i in range(n)])
        else:
            raise ValueError(ks["type"])
    mask = None
    if cfg["op"] == "mask":
        mask = np.stack([G.bernoulli_mask(s["mask"] + i, h, w, cfg["mask_keep"])
                         for i in range(n)])
    elif cfg["op"] == "mri":
        mask = np.stack([G.cartesian_mask(s["mask"] + i, h, w, cfg["accel"], cfg["center"])
                         for i in range(n)])
    ns = cfg["noise_sigma"]
    if isinstance(ns, (list, tuple)):
        rng = np.random.default_rng(s["noise"] + 99991)
        sig = rng.uniform(ns[0], ns[1], n)
        noise = np.stack([G.gaussian_noise(s["noise"] + i, (c, h, w), float(sig[i]))
                          for i in range(n)])
    elif cfg["op"] == "rician":  # real and imaginary noise fields
        noise = np.stack([G.gaussian_noise(s["noise"] + i, (2, c, h, w), ns) for i in range(n)])
    else:
        noise = np.stack([G.gaussian_noise(s["noise"] + i, (c, h, w), ns) for i in range(n)])
    out = dict(x_true=x_true, kern=kern, mask=mask, noise=noise,
               weights=G.init_weights(s["weights"], net_layout(cfg["net"], c)))
    if "warm" in cfg:
        out["warm_weights"] = G.init_weights(s["warm"], G.cnn_layout(cfg["warm"]["chans"]))
    return out
