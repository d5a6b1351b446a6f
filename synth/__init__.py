"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package only draws random numbers and lays them out: ground-truth images,
blur kernels, inpainting masks, noise and network weights.  It holds none of the
method's arithmetic (no forward operator, no network, no iteration), so both sides
can read the same inputs without sharing any computation.
"""
from .generators import (  # noqa: F401
    synth_image,
    synth_batch,
    gaussian_kernel,
    motion_kernel,
    bernoulli_mask,
    gaussian_noise,
    unet_layout,
    cnn_layout,
    init_weights,
)
from .configs import CONFIGS, get_config, workload  # noqa: F401
