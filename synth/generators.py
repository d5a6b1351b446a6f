"""Seeded generators for images, kernels, masks, noise and weights.

Everything is drawn with ``numpy.random.default_rng(seed)`` in float64 and returned
as float32 (uint8 for masks), so that the FP64 oracle and the GPU path start from
bit-identical inputs.  The paper (Sec. 4) evaluates on fastMRI and BSDS500 with
pretrained GS-Denoiser weights; none of that is available here, so these seeded
generators stand in for the images, the degradations and the weights.
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------------------- images

def synth_image(seed: int, c: int, h: int, w: int) -> np.ndarray:
    """One synthetic image in [0,1], shape (c, h, w), float32.

    Piecewise-constant shapes (6 ellipses, 6 rectangles, intensities U[0.2,0.9])
    painted over a mid-grey background, plus a smooth texture of 4 random
    low-frequency cosines (at most 3 cycles across the image, amplitude 0.1).
    Colour images get an independent offset U[-0.1,0.1] per channel.  Clipped to
    [0,1].
    """
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(h) / h, np.arange(w) / w, indexing="ij")
    base = np.full((h, w), 0.5)
    for _ in range(6):  # ellipses
        cy, cx = rng.uniform(0.0, 1.0, 2)
        ry, rx = rng.uniform(0.05, 0.3, 2)
        th = rng.uniform(0.0, math.pi)
        val = rng.uniform(0.2, 0.9)
        dy, dx = yy - cy, xx - cx
        u = (dx * math.cos(th) + dy * math.sin(th)) / rx
        v = (-dx * math.sin(th) + dy * math.cos(th)) / ry
        base[u * u + v * v <= 1.0] = val
    for _ in range(6):  # rectangles
        y0, x0 = rng.uniform(0.0, 0.9, 2)
        hh, ww = rng.uniform(0.05, 0.35, 2)
        val = rng.uniform(0.2, 0.9)
        base[(yy >= y0) & (yy < y0 + hh) & (xx >= x0) & (xx < x0 + ww)] = val
    tex = np.zeros((h, w))
    for _ in range(4):
        fy, fx = rng.uniform(-3.0, 3.0, 2)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        tex += 0.1 * np.cos(2.0 * math.pi * (fy * yy + fx * xx) + ph)
    img = np.empty((c, h, w))
    offs = rng.uniform(-0.1, 0.1, c) if c > 1 else np.zeros(1)
    for ch in range(c):
        img[ch] = base + tex + offs[ch]
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def synth_batch(seed0: int, n: int, c: int, h: int, w: int) -> np.ndarray:
    """n images with seeds seed0 .. seed0+n-1, shape (n, c, h, w), float32."""
    return np.stack([synth_image(seed0 + i, c, h, w) for i in range(n)])


# --------------------------------------------------------------------------- kernels

def gaussian_kernel(size: int, sigma: float) -> np.ndarray:
    """Normalised isotropic Gaussian, shape (size, size), float32 (size odd)."""
    r = size // 2
    ax = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-(ax[:, None] ** 2 + ax[None, :] ** 2) / (2.0 * sigma * sigma))
    return (g / g.sum()).astype(np.float32)


def motion_kernel(seed: int, size: int = 25, steps: int = 64, step: float = 0.5,
                  turn_sd: float = 0.6) -> np.ndarray:
    """Random-walk motion-blur kernel, shape (size, size), float32, sums to 1.

    The walk starts at the centre with a uniform heading, turns by N(0, turn_sd)
    radians per step, advances ``step`` pixels, stays inside the support, and is
    splatted bilinearly into the kernel.
    """
    rng = np.random.default_rng(seed)
    k = np.zeros((size, size))
    py = px = (size - 1) / 2.0
    head = rng.uniform(0.0, 2.0 * math.pi)
    for _ in range(steps):
        iy, ix = int(math.floor(py)), int(math.floor(px))
        fy, fx = py - iy, px - ix
        for dy, wy in ((0, 1.0 - fy), (1, fy)):
            for dx, wx in ((0, 1.0 - fx), (1, fx)):
                yy, xx = min(iy + dy, size - 1), min(ix + dx, size - 1)
                k[yy, xx] += wy * wx
        head += rng.normal(0.0, turn_sd)
        py = min(max(py + step * math.sin(head), 0.0), size - 1.0)
        px = min(max(px + step * math.cos(head), 0.0), size - 1.0)
    return (k / k.sum()).astype(np.float32)


def bernoulli_mask(seed: int, h: int, w: int, keep: float) -> np.ndarray:
    """Per-pixel Bernoulli(keep) inpainting mask, shape (h, w), uint8 in {0,1}."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.0, 1.0, (h, w)) < keep).astype(np.uint8)


def gaussian_noise(seed: int, shape, sigma: float) -> np.ndarray:
    """iid N(0, sigma^2) noise of the given shape, float32."""
    rng = np.random.default_rng(seed)
    return (sigma * rng.standard_normal(shape)).astype(np.float32)


# --------------------------------------------------------------------------- weights
#
# Flat weight-vector formats.  Each entry is (name, kind, shape, fan_in, gain):
#   kind "conv3": 3x3 convolution, shape (C_out, C_in, 3, 3)
#   kind "down" : 2x2 stride-2 convolution, shape (C_out, C_in, 2, 2)
#   kind "up"   : 2x2 stride-2 transposed convolution, shape (C_in, C_out, 2, 2)
# Tensors are concatenated in list order, each in C order.  Weights are drawn
# N(0, gain^2 * v / fan_in), v = 2 (He) in front of an activation, else 1.

def unet_layout(c: int, widths, n_rb: int = 2):
    """Weight list of the 4-scale residual U-Net regulariser.

    head 3x3 c->w0; per encoder level l<L-1: n_rb residual blocks
    (3x3 conv, softplus, 3x3 conv, identity skip) then a 2x2 stride-2 conv
    w_l -> w_{l+1}; n_rb blocks at the coarsest level; per decoder level
    (coarse to fine): 2x2 stride-2 transposed conv w_{l+1} -> w_l, add the
    encoder output of that level, n_rb blocks; tail 3x3 w0 -> c.  No biases.
    """
    L = len(widths)
    out = [("head", "conv3", (widths[0], c, 3, 3), 9 * c, 1.0, 1.0)]

    def rbs(prefix, wd):
        for r in range(n_rb):
            out.append((f"{prefix}.rb{r}.c1", "conv3", (wd, wd, 3, 3), 9 * wd, 2.0, 1.0))
            out.append((f"{prefix}.rb{r}.c2", "conv3", (wd, wd, 3, 3), 9 * wd, 2.0, 0.1))

    for lv in range(L - 1):
        rbs(f"enc{lv}", widths[lv])
        out.append((f"enc{lv}.down", "down", (widths[lv + 1], widths[lv], 2, 2),
                    4 * widths[lv], 1.0, 1.0))
    rbs(f"mid{L - 1}", widths[L - 1])
    for lv in range(L - 2, -1, -1):
        out.append((f"dec{lv}.up", "up", (widths[lv + 1], widths[lv], 2, 2),
                    widths[lv + 1], 1.0, 1.0))
        rbs(f"dec{lv}", widths[lv])
    out.append(("tail", "conv3", (c, widths[0], 3, 3), 9 * widths[0], 1.0, 0.1))
    return out


def cnn_layout(chans, last_gain: float = 0.1):
    """Weight list of a plain 3x3 conv stack chans[0] -> ... -> chans[-1].

    An activation follows every layer but the last; the last layer's weights
    are scaled by ``last_gain``.
    """
    out = []
    n = len(chans) - 1
    for i in range(n):
        last = i == n - 1
        out.append((f"l{i}", "conv3", (chans[i + 1], chans[i], 3, 3), 9 * chans[i],
                    1.0 if last else 2.0, last_gain if last else 1.0))
    return out


def init_weights(seed: int, layout) -> np.ndarray:
    """Flat float32 weight vector for ``layout``, seeded He/LeCun-normal init."""
    rng = np.random.default_rng(seed)
    parts = []
    for (_name, _kind, shape, fan_in, v, gain) in layout:
        std = gain * math.sqrt(v / fan_in)
        parts.append((std * rng.standard_normal(int(np.prod(shape)))).ravel())
    return np.concatenate(parts).astype(np.float32)


def complex_image(seed: int, h: int, w: int) -> np.ndarray:
    """Complex MR-like image as (re, im) planes (2, h, w): the grey synthetic image
    as magnitude times a smooth phase exp(i phi), phi a sum of 3 low-frequency
    cosines (<= 2 cycles) of amplitude <= 0.5 rad."""
    mag = synth_image(seed, 1, h, w)[0].astype(np.float64)
    rng = np.random.default_rng(seed + 777)
    yy, xx = np.meshgrid(np.arange(h) / h, np.arange(w) / w, indexing="ij")
    phi = np.zeros((h, w))
    for _ in range(3):
        fy, fx = rng.integers(0, 3, 2)
        phi += rng.uniform(0.0, 0.5 / 3) * np.cos(2 * np.pi * (fy * yy + fx * xx) +
                                                 rng.uniform(0, 2 * np.pi))
    return np.stack([mag * np.cos(phi), mag * np.sin(phi)]).astype(np.float32)


def cartesian_mask(seed: int, h: int, w: int, accel: int = 4, center: float = 0.08) -> np.ndarray:
    """Cartesian k-space sampling (h, w) u8 in the unshifted FFT layout: whole
    columns (phase-encoding lines), the centre fraction around frequency 0 always
    sampled and the rest drawn uniformly until w / accel columns are taken."""
    rng = np.random.default_rng(seed)
    n_keep = max(1, w // accel)
    n_c = max(1, int(round(center * w)))
    freqs = np.fft.fftfreq(w) * w  # integer frequency of each column
    order = np.argsort(np.abs(freqs), kind="stable")
    cols = set(order[:n_c].tolist())
    rest = [c for c in range(w) if c not in cols]
    extra = rng.choice(rest, size=max(0, n_keep - len(cols)), replace=False)
    cols.update(int(c) for c in extra)
    m = np.zeros((h, w), dtype=np.uint8)
    m[:, sorted(cols)] = 1
    return m
