"""What the trained denoiser gains over the method without it (App. C).

The committed network was trained on the GPU by the library's own kernels at
the noise level sigma that the heuristic sets for the 4096^2 workload
(Eq. sigma).  On held-out synthetic skies (a seed the training never used)
corrupted at that sigma, its output is compared with the two denoisers the
method has without it: positivity alone (the identity of the residual form)
and the one-level Haar soft threshold at t = sigma with positivity, the plain
loop's prox at this noise level (App. B, Eq. lambda).  Errors are mean |D(z) -
u| over the images, the quantity the network was trained to lower.
"""
import os

import numpy as np
import pytest

import synth

from gpu_common import pnp, require_gpu, to_dev_f32, to_host, torch

pytestmark = pytest.mark.gpu
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2207_11336_gb300",
                       "weights", "dncnn_C3.npz")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_trained_denoiser_beats_positivity_and_haar_at_its_noise_level():
    from paper_2207_11336_gb300.train_denoiser import load
    params, meta = load(WEIGHTS)
    sigma = float(meta["sigma"])
    n, count = 256, 6
    rng = np.random.default_rng(20260)             # held out: training used SeedSequence([0, 0x7A11])
    cnn = pnp.CnnDenoiser(params, n, halo=0)
    haar = pnp.HaarDenoiser(sigma)
    err = {"positivity": 0.0, "haar": 0.0, "cnn": 0.0}
    for _ in range(count):
        u = synth.training_image(n, rng)
        z = u + sigma * rng.standard_normal((n, n))
        zd = to_dev_f32(z)
        err["positivity"] += np.abs(np.maximum(z, 0.0) - u).mean() / count
        err["haar"] += np.abs(to_host(haar.denoise(zd)) - u).mean() / count
        err["cnn"] += np.abs(to_host(cnn.denoise(zd)) - u).mean() / count
    print({k: f"{v:.3e}" for k, v in err.items()}, "sigma", sigma)
    assert cnn.device_status() == 0
    assert err["cnn"] < 0.5 * err["positivity"]
    assert err["cnn"] < err["haar"]
