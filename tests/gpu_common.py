"""Shared set-up of the GPU parity tests: seeded inputs, oracle objects, C-ABI contexts."""
from __future__ import annotations

import numpy as np

from oracle import nets, operators
from synth import get_config, workload


def setup(name, **over):
    """(cfg, workload, oracle net, oracle operators, y as float32).

    y = A(x*) + n is formed by the oracle in FP64 and rounded to float32; both
    sides then start from the same float32 observations."""
    cfg = get_config(name, **over)
    wl = workload(cfg)
    net = nets.Net.from_config(cfg["net"], cfg["c"], wl["weights"])
    ops = operators.make_operators(cfg, wl)
    ys = operators.observe(ops, wl["x_true"], wl["noise"]).astype(np.float32)
    return cfg, wl, net, ops, ys


def ctx_for(cfg, wl, precision):
    import torch
    from paper_2605_19705_gb300 import binding as B
    desc = B.net_desc(cfg["net"], cfg["c"])
    w = torch.tensor(wl["weights"], device="cuda")
    return B.Context(desc, w, precision)


def op_for(cfg, wl):
    import torch
    from paper_2605_19705_gb300 import binding as B
    kind = {"blur": B.IDEQ_OP_BLUR, "mask": B.IDEQ_OP_MASK, "satblur": B.IDEQ_OP_SATBLUR,
            "mri": B.IDEQ_OP_MRI, "rician": B.IDEQ_OP_RICIAN}[cfg["op"]]
    kern = None if wl["kern"] is None else torch.tensor(wl["kern"], device="cuda").contiguous()
    mask = None if wl["mask"] is None else torch.tensor(wl["mask"], device="cuda").contiguous()
    sigma = cfg["noise_sigma"] if cfg["op"] == "rician" else 0.0
    return B.make_operator(kind, kern, mask, cfg.get("sat_gain", 2.0), sigma)


def rel(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_np(t):
    return t.detach().double().cpu().numpy()
