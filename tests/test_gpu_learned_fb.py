"""The learned PnP-FB loop (App. C, F) on the GPU against the FP64 learned oracle.

A 64^2 image / 128^2 grid / M = 1.5e4 problem of the 256^2 configuration's kind (KB rows, no w,
40 dB input SNR) with Briggs-weighted data (robust 0, Sec. 3), the committed trained network on
2 x 2 facets with a 32 px halo, and 120 iterations of Eq. fb on both sides.  The problem is
rescaled through pnp_fb_run's alpha (App. C, Eq. invpb2) by the larger of the dirty-peak bound
max(Re{Phi^H y}) / beta and the alpha that matches the data to the network's training noise
level (Eq. sigma, App. F).  The GPU runs the FP32 operator and the BF16 network; the oracle runs
FP64 throughout.  The weighting puts the reconstruction well above 0 dB; the SNRs must agree
within 0.5 dB, and the images closely.
"""
import os

import numpy as np
import pytest

import synth
from oracle import cnn as ocnn
from oracle import fb as ofb
from oracle import nufft as onu

from gpu_common import pnp, rel_l2, require_gpu, to_dev_c64, to_host

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2207_11336_gb300", "weights", "dncnn_C3.npz")


def test_learned_loop_snr_matches_fp64_oracle():
    require_gpu()
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained weights")
    from paper_2207_11336_gb300.train_denoiser import load
    params, meta = load(WEIGHTS)
    n, K, M, iters = 64, 128, 15000, 120
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    d = np.sqrt(synth.briggs_weights(prob["omega"], n, 0.0))
    ora = onu.Operator(n, K, prob["omega"], row_scale=d)
    y_raw = onu.Operator(n, K, prob["omega"]).forward(prob["x_true"])
    tau = synth.noise_std_for_isnr(np.linalg.norm(y_raw), M, prob["isnr_db"])
    y = d * (y_raw + tau * prob["noise"])
    tau_w = tau * np.sqrt(np.mean(d ** 2))
    L, _, _ = ofb.power_iteration(ora, synth.rng_for("power").standard_normal((n, n)), 1000, 1e-10)
    gamma = ofb.step_size(L)
    alpha = max(ofb.dirty_peak(ora, y, ofb.psf_peak(ora)), ofb.alpha_for_denoiser(tau_w, L, float(meta["sigma"])))
    x_ref, h = ofb.pnp_fb(ora, y, gamma, lambda z: ocnn.denoise(params, z), iters, x_true=prob["x_true"],
                          alpha=alpha)
    plan = pnp.Plan(n, K, prob["omega"], row_scale=d)
    den = pnp.CnnDenoiser(params, n, facet_rows=[32, 32], facet_cols=[32, 32], halo=32)
    x, st = plan.fb_run(den, to_dev_c64(y), gamma=gamma, L=L, max_iter=iters, check_every=10, alpha=alpha)
    assert st.iters == iters and den.device_status() == 0
    xg = to_host(x)
    snr_gpu = ofb.snr_db(prob["x_true"], xg)
    snr_ref = ofb.snr_db(prob["x_true"], x_ref)
    print(f"learned loop SNR after {iters} iterations (alpha {alpha:.3g}): GPU {snr_gpu:.3f} dB, "
          f"FP64 oracle {snr_ref:.3f} dB")
    assert snr_ref > 3.0
    assert abs(snr_gpu - snr_ref) <= 0.5
    assert rel_l2(xg, x_ref) <= 2e-2
