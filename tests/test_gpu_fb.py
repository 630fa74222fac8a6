"""GPU parity of the plain PnP-FB loop (Eq. fb with the Haar prox of App. B) vs the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import fb as ofb
from oracle import nufft as onu

from gpu_common import pnp, rel_l2, require_gpu, to_dev_c64, to_dev_f32, to_host, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _c0_like(n, K, M):
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    ora = onu.Operator(n, K, prob["omega"])
    y0 = ora.forward(prob["x_true"])
    tau = synth.noise_std_for_isnr(np.linalg.norm(y0), M, prob["isnr_db"])
    y = y0 + tau * prob["noise"]
    return prob, ora, y, tau


def test_haar_denoiser_parity():
    rng = np.random.default_rng(3)
    z = rng.standard_normal((66, 66)).astype(np.float32).astype(np.float64)
    den = pnp.HaarDenoiser(0.3)
    out = to_host(den.denoise(to_dev_f32(z)))
    assert np.allclose(out, ofb.haar_denoise(z, 0.3), atol=1e-6)


@pytest.mark.parametrize("n,K,M,iters", [(64, 128, 20000, 60), (256, 512, 200000, 200)])
def test_plain_pnp_fb_parity(n, K, M, iters):
    """200 iterations of the 256^2 / M = 2e5 plain loop: final image rel. L2 <= 1e-4."""
    prob, ora, y, tau = _c0_like(n, K, M)
    v0 = synth.rng_for("power").standard_normal((n, n))
    L, _, _ = ofb.power_iteration(ora, v0, 1000, 1e-10)
    gamma = ofb.step_size(L)
    t = ofb.soft_threshold_from_noise(tau, L)
    x_ref, _ = ofb.pnp_fb(ora, y, gamma, lambda z: ofb.haar_denoise(z, t), iters)
    plan = pnp.Plan(n, K, prob["omega"])
    den = pnp.HaarDenoiser(t)
    x, st = plan.fb_run(den, to_dev_c64(y), gamma=gamma, L=L, max_iter=iters, check_every=10)
    assert st.iters == iters
    assert rel_l2(to_host(x), x_ref) <= 1e-4
    # the reconstruction improves on the dirty start
    assert ofb.snr_db(prob["x_true"], x_ref) > 0


def test_graph_and_eager_agree_and_tol_stops():
    n, K, M = 64, 128, 20000
    prob, ora, y, tau = _c0_like(n, K, M)
    plan = pnp.Plan(n, K, prob["omega"])
    L, _ = plan.op_norm(None, 500, 1e-7)
    den = pnp.HaarDenoiser(ofb.soft_threshold_from_noise(tau, L))
    yd = to_dev_c64(y)
    xa, sa = plan.fb_run(den, yd, L=L, max_iter=41, check_every=10, use_graph=True)
    xb, sb = plan.fb_run(den, yd, L=L, max_iter=41, check_every=10, use_graph=False)
    assert sa.iters == sb.iters == 41
    assert rel_l2(to_host(xa), to_host(xb)) <= 1e-5
    xc, sc = plan.fb_run(den, yd, L=L, max_iter=1000, tol=1e-3, check_every=2)
    assert sc.iters < 1000 and sc.rel_change < 1e-3


def test_grad_step_then_denoise_equals_one_fb_iteration():
    n, K, M = 64, 128, 20000
    prob, ora, y, tau = _c0_like(n, K, M)
    plan = pnp.Plan(n, K, prob["omega"])
    L, _ = plan.op_norm(None, 500, 1e-7)
    den = pnp.HaarDenoiser(0.01)
    x0 = to_dev_f32(prob["x_true"])
    yd = to_dev_c64(y)
    z = plan.grad_step(x0, yd, 1.98 / L)
    x1 = to_host(den.denoise(z))
    x2, _ = plan.fb_run(den, yd, x0=x0, L=L, max_iter=1, use_graph=False)
    assert rel_l2(to_host(x2), x1) <= 1e-6


def test_divergence_is_reported():
    # fault injected on the host: a non-finite visibility makes the iterate non-finite,
    # which the FP64 stopping-test norms detect
    n, K, M = 32, 64, 5000
    prob, ora, y, tau = _c0_like(n, K, M)
    plan = pnp.Plan(n, K, prob["omega"])
    den = pnp.HaarDenoiser(0.0)
    L, _ = plan.op_norm(None, 500, 1e-7)
    y_bad = y.copy()
    y_bad[17] = np.nan
    with pytest.raises(pnp.PnPError) as ei:
        plan.fb_run(den, to_dev_c64(y_bad), L=L, max_iter=20, check_every=4)
    assert ei.value.code == -4
    # the plan stays usable afterwards
    x, st = plan.fb_run(den, to_dev_c64(y), L=L, max_iter=4, check_every=4)
    assert st.iters == 4 and np.isfinite(to_host(x)).all()
