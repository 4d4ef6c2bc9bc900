"""MM-RSMoE denoising (Sec. V-C): H R-SMoE models of one noisy image, fitted
together as one ragged batch (one binning, one fused tile launch and one
Adam launch per iteration for all H), then fused by the per-pixel mean of
their renders (Eq. 11) in one launch.

The H models differ by the block window they start from: the window is
shifted horizontally and vertically by multiples of a displacement d, and
each model's initial kernel lattice moves with its window (its own jitter
seed as well).  With the per-pixel truncation q <= q_max the fitted function
does not depend on where the tile grid lies, so the shift acts through the
initial lattice; each model's different start is what gives it the
independent "model noise" of Eq. 10 that the averaging of Eq. 11-14 removes.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import synth
from .api import SMoEParams
from .fit import FitBatch


def shift_offsets(n_models: int, block: int = 16):
    """Window offsets (ox, oy) in pixels for n_models shifted windows of a
    block x block window: displacement d = block / n per axis gives
    n_x * n_y = n_models models, (block/d)^2 for a square count (d = 2, 4, 8,
    16 -> 64, 16, 4, 1 models for 16-pixel blocks); a count that is twice a
    square takes twice the offsets along x (8 -> 4 x 2, 32 -> 8 x 4)."""
    if n_models < 1:
        raise ValueError("n_models must be >= 1")
    r = math.isqrt(n_models)
    if r * r == n_models:
        nx = ny = r
    elif n_models % 2 == 0 and math.isqrt(n_models // 2) ** 2 == n_models // 2:
        ny = math.isqrt(n_models // 2)
        nx = 2 * ny
    else:
        nx, ny = n_models, 1
    if block % nx or block % ny:
        raise ValueError(f"{n_models} windows do not divide a {block}-pixel block evenly")
    dx, dy = block // nx, block // ny
    return [(i * dx, j * dy) for j in range(ny) for i in range(nx)]


def init_models(noisy: np.ndarray, n_models: int, K: int, sigma: float = 5.0,
                linear: bool = True, seed: int = 0, block: int = 16):
    """The H initial models: K kernels each on the jittered lattice shifted
    by the model's window offset, bandwidth sigma px, experts from the noisy
    image at the nearest pixel."""
    return [SMoEParams.from_numpy(synth.init_params(noisy, K, sigma, linear, seed + h,
                                                    offset=off))
            for h, off in enumerate(shift_offsets(n_models, block))]


def mm_rsmoe(noisy: torch.Tensor, models, iters: int, lr=None, tile: int = 16,
             qmax: float = 9.0, graph_iters: int | None = None, deterministic: bool = False,
             persistent: bool = False):
    """Fit the H models (list of SMoEParams, updated in place) to the one
    noisy (C, H, W) CUDA image for `iters` iterations and return the fused
    prediction y_m (C, H, W) and the FitBatch (for losses and parameters).
    The H images of the batch share the one target tensor."""
    fb = FitBatch([noisy] * len(models), list(models), iters, lr=lr, tile=tile, qmax=qmax,
                  deterministic=deterministic, persistent=persistent)
    fb.run(iters, graph_iters=graph_iters)
    return fb.render_mean(), fb
