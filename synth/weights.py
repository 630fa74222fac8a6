"""Seeded initial weights for the residual CNN denoiser (He-normal, zero bias)."""
from __future__ import annotations

import numpy as np


def cnn_init(rng: np.random.Generator, channels: int = 64, depth: int = 8, last_scale: float = 0.1):
    """List of (W (co, ci, 3, 3) float64, b (co,) float64) for 1 -> C -> ... -> C -> 1.

    Hidden layers use He-normal std sqrt(2 / (9 ci)); the last layer is scaled
    by ``last_scale`` so the untrained residual starts close to the identity.
    """
    shapes = [(channels, 1)] + [(channels, channels)] * (depth - 2) + [(1, channels)]
    out = []
    for i, (co, ci) in enumerate(shapes):
        std = np.sqrt(2.0 / (9.0 * ci)) * (last_scale if i == depth - 1 else 1.0)
        out.append((rng.normal(0.0, std, (co, ci, 3, 3)), np.zeros(co)))
    return out
