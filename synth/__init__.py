"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds input generation only: antenna layouts, uv tracks, sky
models, noise draws, block and facet layouts.  It contains none of the
imaging method's arithmetic (no kernels, no Fourier transforms, no operator),
so both the FP64 oracle and the CUDA path can consume the same arrays without
sharing any code that computes a result.

The real MeerKAT observation of ESO 137-006 used in the paper (Sec. 3) is not
available; these MeerKAT-like arrays stand in for its shapes: 64 antennas,
baselines up to ~8 km, L band, a southern declination.
"""
from .meerkat import (  # noqa: F401
    SEED_STREAMS, rng_for, antenna_layout, uvw_track, imaging_geometry,
    j_per_row_by_w_quartile, sky_model, training_image, complex_normal,
    noise_std_for_isnr, radial_blocks, facet_layout, w_stacks, w_stacks_min_taps,
    j_per_row_stacked, briggs_weights,
)
from .configs import CONFIGS, make_problem  # noqa: F401
from .weights import cnn_init  # noqa: F401,E402
