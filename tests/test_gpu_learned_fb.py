"""The learned PnP-FB loop (App. C, F) on the GPU against the FP64 learned oracle.

A 96^2 image / 256^2 grid / M = 3e4 problem of the 256^2 configuration's kind (KB rows, no w,
40 dB input SNR), the committed trained network on 2 x 2 facets with a 32 px halo, the problem
rescaled by alpha = max(Re{Phi^H y}) / beta (App. F) and 30 iterations of Eq. fb on both sides.
The GPU runs the FP32 operator and the BF16 network; the oracle runs FP64 throughout.  The
reconstruction SNRs must agree within 0.5 dB, and the images closely.
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
    params, _ = load(WEIGHTS)
    n, K, M, iters = 96, 256, 30000, 30
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    ora = onu.Operator(n, K, prob["omega"])
    y0 = ora.forward(prob["x_true"])
    tau = synth.noise_std_for_isnr(np.linalg.norm(y0), M, prob["isnr_db"])
    y = y0 + tau * prob["noise"]
    L, _, _ = ofb.power_iteration(ora, synth.rng_for("power").standard_normal((n, n)), 1000, 1e-10)
    gamma = ofb.step_size(L)
    alpha = ofb.dirty_peak(ora, y, ofb.psf_peak(ora))
    ys = y / alpha
    x_ref, _ = ofb.pnp_fb(ora, ys, gamma, lambda z: ocnn.denoise(params, z), iters)
    plan = pnp.Plan(n, K, prob["omega"])
    den = pnp.CnnDenoiser(params, n, facet_rows=[48, 48], facet_cols=[48, 48], halo=32)
    x, st = plan.fb_run(den, to_dev_c64(ys), gamma=gamma, L=L, max_iter=iters, check_every=10)
    assert st.iters == iters and den.device_status() == 0
    xg = to_host(x)
    snr_gpu = ofb.snr_db(prob["x_true"], alpha * xg)
    snr_ref = ofb.snr_db(prob["x_true"], alpha * x_ref)
    print(f"learned loop SNR after {iters} iterations: GPU {snr_gpu:.3f} dB, FP64 oracle {snr_ref:.3f} dB")
    assert abs(snr_gpu - snr_ref) <= 0.5
    assert rel_l2(xg, x_ref) <= 2e-2
