"""Independent PyTorch (CPU, float64) restatement of the regulariser networks.

Used only to pin the oracle: the architecture is written out directly with
torch.nn.functional calls (not by interpreting the oracle's op list) and
torch.autograd supplies every derivative, so that a wrong skip, index, sign or
transpose in the oracle's hand-derived passes shows up as a mismatch.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F


def unpack(flat, layout):
    """Split a flat weight vector by a synth layout into named tensors."""
    flat = torch.as_tensor(np.asarray(flat, dtype=np.float64))
    out, off = {}, 0
    for name, _kind, shape, *_ in layout:
        n = int(np.prod(shape))
        out[name] = flat[off:off + n].reshape(shape).clone()
        off += n
    assert off == flat.numel()
    return out


def unet(W, x, widths, n_rb=2):
    """x: (B, c, h, w).  The residual U-Net described in synth.unet_layout."""
    L = len(widths)

    def rbs(prefix, h):
        for r in range(n_rb):
            t = F.conv2d(h, W[f"{prefix}.rb{r}.c1"], padding=1)
            h = h + F.conv2d(F.softplus(t), W[f"{prefix}.rb{r}.c2"], padding=1)
        return h

    h = F.conv2d(x, W["head"], padding=1)
    skips = []
    for lv in range(L - 1):
        h = rbs(f"enc{lv}", h)
        skips.append(h)
        h = F.conv2d(h, W[f"enc{lv}.down"], stride=2)
    h = rbs(f"mid{L - 1}", h)
    for lv in range(L - 2, -1, -1):
        h = F.conv_transpose2d(h, W[f"dec{lv}.up"], stride=2) + skips[lv]
        h = rbs(f"dec{lv}", h)
    return F.conv2d(h, W["tail"], padding=1)


def cnn(W, x, n_layers, act="softplus"):
    a = F.softplus if act == "softplus" else F.relu
    h = x
    for i in range(n_layers):
        h = F.conv2d(h, W[f"l{i}"], padding=1)
        if i < n_layers - 1:
            h = a(h)
    return h


def g_of(netfn, x):
    """g(x) = 1/2 ||x - N(x)||^2 for a batch of one."""
    r = x - netfn(x)
    return 0.5 * (r * r).sum()
