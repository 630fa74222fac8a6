"""GPU uSARA denoiser (App. B) against the SARA oracle: dictionary, prox, reweighting, FB loop."""
import numpy as np
import pytest

import synth
from oracle import fb as ofb
from oracle import nufft as onu
from oracle import sara as osa

from gpu_common import pnp, rel_l2, require_gpu, to_dev_c64, to_dev_f32, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("n,levels", [(64, 4), (96, 4), (48, 4), (1024, 4), (512, 6)])
def test_sara_dictionary_matches_oracle(n, levels):
    """Psi^T and Psi against the oracle: coarse levels shorter than the db8 filter (48 / 8 = 6 < 16),
    a side that is not a power of two, and sides that span several tiles of the DWT passes."""
    x = np.random.default_rng(1).standard_normal((n, n))
    den = pnp.SaraDenoiser(n, 0.1, 0.1, 1, levels=levels)
    c = to_host(den.analysis(to_dev_f32(x)))
    psi = osa.Sara(levels=levels)
    ref = psi.analysis(x)
    assert rel_l2(c, ref) <= 1e-6
    back = to_host(den.synthesis(to_dev_f32(ref.astype(np.float32))))
    assert rel_l2(back, psi.synthesis(ref.astype(np.float32).astype(np.float64))) <= 1e-6


@pytest.mark.parametrize("reweight", [False, True])
def test_sara_prox_matches_oracle(reweight):
    n, gl, iters = 64, 0.05, 25
    rng = np.random.default_rng(2)
    z = rng.standard_normal((n, n)) + 0.3
    den = pnp.SaraDenoiser(n, gl, gl, iters, levels=4)
    psi = osa.Sara(levels=4)
    w = np.ones((9, n, n))
    if reweight:
        xw = np.maximum(rng.standard_normal((n, n)), 0).astype(np.float32)
        den.reweight(to_dev_f32(xw))
        w = osa.reweighting_weights(psi.analysis(xw.astype(np.float64)), gl)
    x = to_host(den.denoise(to_dev_f32(z)))
    ref, _, _ = osa.prox_weighted_l1_pos(psi, z.astype(np.float32).astype(np.float64), gl * w, iters, 0.0)
    assert rel_l2(x, ref) <= 1e-5


def test_usara_fb_loop_matches_oracle():
    n, K, M, iters, prox_iters = 64, 128, 20000, 8, 10
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    ora = onu.Operator(n, K, prob["omega"])
    y0 = ora.forward(prob["x_true"])
    tau = synth.noise_std_for_isnr(np.linalg.norm(y0), M, prob["isnr_db"])
    y = y0 + tau * prob["noise"]
    L, _, _ = ofb.power_iteration(ora, synth.rng_for("power").standard_normal((n, n)), 1000, 1e-10)
    gamma = ofb.step_size(L)
    gl = ofb.soft_threshold_from_noise(tau, L)
    x_ref = osa.usara(ora, y, gamma, gl, gl, 0, iters, prox_iters=prox_iters, psi=osa.Sara(levels=4),
                      prox_tol=0.0)
    plan = pnp.Plan(n, K, prob["omega"])
    den = pnp.SaraDenoiser(n, gl, gl, prox_iters, levels=4)
    x, st = plan.fb_run(den, to_dev_c64(y), gamma=gamma, L=L, max_iter=iters, check_every=4)
    assert st.iters == iters
    assert rel_l2(to_host(x), x_ref) <= 1e-4


def test_reweighted_usara_inside_pnp_fb_run_matches_oracle():
    """uSARA as App. B runs it: three weighted-l1 surrogates of 4 FB iterations each, the weights
    re-formed from the iterate by pnp_fb_run itself (reweight_every), against the oracle's loop."""
    n, K, M, fb_iters, prox_iters = 64, 128, 20000, 4, 10
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    ora = onu.Operator(n, K, prob["omega"])
    y0 = ora.forward(prob["x_true"])
    tau = synth.noise_std_for_isnr(np.linalg.norm(y0), M, prob["isnr_db"])
    y = y0 + tau * prob["noise"]
    L, _, _ = ofb.power_iteration(ora, synth.rng_for("power").standard_normal((n, n)), 1000, 1e-10)
    gamma = ofb.step_size(L)
    gl = ofb.soft_threshold_from_noise(tau, L)
    x_ref = osa.usara(ora, y, gamma, gl, gl, 2, fb_iters, prox_iters=prox_iters, psi=osa.Sara(levels=4),
                      prox_tol=0.0)
    plan = pnp.Plan(n, K, prob["omega"])
    den = pnp.SaraDenoiser(n, gl, gl, prox_iters, levels=4)
    x, st = plan.fb_run(den, to_dev_c64(y), gamma=gamma, L=L, max_iter=3 * fb_iters, check_every=10,
                        reweight_every=fb_iters)
    assert st.iters == 3 * fb_iters
    assert rel_l2(to_host(x), x_ref) <= 1e-4
    # the same run without reweighting differs (the weights matter), and a Haar denoiser refuses it
    den2 = pnp.SaraDenoiser(n, gl, gl, prox_iters, levels=4)
    x_plain, _ = plan.fb_run(den2, to_dev_c64(y), gamma=gamma, L=L, max_iter=3 * fb_iters, check_every=10)
    assert rel_l2(to_host(x_plain), x_ref) > 1e-4
    with pytest.raises(pnp.PnPError):
        plan.fb_run(pnp.HaarDenoiser(0.1), to_dev_c64(y), L=L, max_iter=2, reweight_every=1)
