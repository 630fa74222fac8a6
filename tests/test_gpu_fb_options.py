"""GPU parity of the PnP-FB options behind the C ABI: data weights on the rows of G (Sec. 3, Briggs
weighting), the App. C rescaling by alpha (Eq. invpb2), the positivity switch, the learned -> plain
fallback (App. C) and the CUDA graph kept across pnp_fb_run calls."""
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


def _weighted(n=64, K=128, M=15000):
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    d = np.sqrt(synth.briggs_weights(prob["omega"], n, 0.0))
    ora = onu.Operator(n, K, prob["omega"], row_scale=d)
    y_raw = onu.Operator(n, K, prob["omega"]).forward(prob["x_true"])
    tau = synth.noise_std_for_isnr(np.linalg.norm(y_raw), M, prob["isnr_db"])
    y_raw = y_raw + tau * prob["noise"]
    return prob, d, ora, y_raw, tau


def test_weighted_operator_matches_oracle():
    prob, d, ora, y_raw, _ = _weighted()
    n, K = prob["n"], prob["K"]
    plan = pnp.Plan(n, K, prob["omega"], row_scale=d)
    x = to_dev_f32(prob["x_true"])
    assert rel_l2(to_host(plan.phi_forward(x)), ora.forward(prob["x_true"])) <= 1e-5
    yw = plan.scale_data(to_dev_c64(y_raw))
    assert rel_l2(to_host(yw), d * y_raw) <= 1e-6
    assert rel_l2(to_host(plan.phi_adjoint(yw)), ora.adjoint(d * y_raw)) <= 1e-5
    # the weighted dirty beam peak is sum_m d_m^2
    delta = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    delta[n // 2, n // 2] = 1.0
    assert float(plan.phi_adjoint(plan.phi_forward(delta)).max()) == pytest.approx(np.sum(d ** 2), rel=1e-5)
    with pytest.raises(pnp.PnPError):
        bad = d.copy()
        bad[3] = 0.0
        pnp.Plan(n, K, prob["omega"], row_scale=bad)


@pytest.mark.parametrize("positivity", [True, False])
def test_alpha_rescaled_weighted_haar_loop_matches_oracle(positivity):
    """pnp_fb_run with alpha != 1 on Briggs-weighted data against the oracle's rescaled loop."""
    prob, d, ora, y_raw, tau = _weighted()
    n, K, iters = prob["n"], prob["K"], 120
    yw = d * y_raw
    L, _, _ = ofb.power_iteration(ora, synth.rng_for("power").standard_normal((n, n)), 2000, 1e-10)
    gamma = ofb.step_size(L)
    alpha = 13.7
    t = ofb.soft_threshold_from_noise(tau * np.sqrt(np.mean(d ** 2)), L) / alpha   # rescaled units
    x_ref, h = ofb.pnp_fb(ora, yw, gamma, lambda z: ofb.haar_denoise(z, t, positivity), iters,
                          x_true=prob["x_true"], alpha=alpha)
    plan = pnp.Plan(n, K, prob["omega"], row_scale=d)
    x, st = plan.fb_run(pnp.HaarDenoiser(t), to_dev_c64(yw), gamma=gamma, L=L, max_iter=iters, check_every=10,
                        alpha=alpha, positivity=positivity)
    xg = to_host(x)
    assert st.iters == iters and st.fallback_iter == -1
    assert rel_l2(xg, x_ref) <= 1e-4
    assert xg.min() >= 0 if positivity else xg.min() < 0
    if positivity:
        assert h["snr"][-1] > 3.0   # Briggs weighting: a regime well above 0 dB


def test_graph_kept_across_calls_and_rebuilt_after_a_work_list_change():
    prob, d, ora, y_raw, tau = _weighted()
    n, K = prob["n"], prob["K"]
    plan = pnp.Plan(n, K, prob["omega"], row_scale=d)
    yw = plan.scale_data(to_dev_c64(y_raw))
    L, _ = plan.op_norm(None, 500, 1e-8)
    den = pnp.HaarDenoiser(1e-3)
    x_one, _ = plan.fb_run(den, yw, L=L, max_iter=40, check_every=40, use_graph=False)
    x = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    for _ in range(4):   # chunks of 10 replay one graph captured by the first chunk
        plan.fb_run(den, yw, x0=x, L=L, max_iter=10, check_every=10, inplace=True)
    assert rel_l2(to_host(x), to_host(x_one)) <= 1e-5
    plan.set_row_batch(1 if plan.info["row_batch"] != 1 else 2)
    plan.set_unit_nnz(1 << 16)
    x.zero_()
    for _ in range(4):
        plan.fb_run(den, yw, x0=x, L=L, max_iter=10, check_every=10, inplace=True)
    assert rel_l2(to_host(x), to_host(x_one)) <= 1e-5


def _amplifying_network(c=1.0):
    """A CNN with N(z) = -c z for z >= 0 (identity paths through channel 0, last layer -c), so that
    D(z) = max(0, (1 + c) z): a learned denoiser that makes the loop diverge (a host-made fault)."""
    params = []
    shapes = [(64, 1)] + [(64, 64)] * 6 + [(1, 64)]
    for li, (co, ci) in enumerate(shapes):
        W = np.zeros((co, ci, 3, 3))
        W[0, 0, 1, 1] = -c if li == len(shapes) - 1 else 1.0
        params.append((W, np.zeros(co)))
    return params


def test_learned_loop_falls_back_to_the_plain_loop_on_divergence():
    prob, d, ora, y_raw, tau = _weighted()
    n, K = prob["n"], prob["K"]
    plan = pnp.Plan(n, K, prob["omega"], row_scale=d)
    yw = plan.scale_data(to_dev_c64(y_raw))
    L, _ = plan.op_norm(None, 500, 1e-8)
    t = ofb.soft_threshold_from_noise(tau * np.sqrt(np.mean(d ** 2)), L)
    cnn = pnp.CnnDenoiser(_amplifying_network(), n, halo=8)
    with pytest.raises(pnp.PnPError) as ei:
        plan.fb_run(cnn, yw, L=L, max_iter=60, check_every=5, diverge_factor=20.0)
    assert ei.value.code == -4
    x, st = plan.fb_run(cnn, yw, L=L, max_iter=60, check_every=5, diverge_factor=20.0, fallback_t=t)
    assert st.iters == 60 and st.fallback_iter >= 5 and st.fallback_iter % 5 == 0
    xg = to_host(x)
    assert np.isfinite(xg).all()
    # the same two stages run by hand: the learned loop to the checkpoint, then the plain loop
    xa, _ = plan.fb_run(cnn, yw, L=L, max_iter=st.fallback_iter, check_every=5, use_graph=False)
    xb, _ = plan.fb_run(pnp.HaarDenoiser(t), yw, x0=xa, L=L, max_iter=60 - st.fallback_iter, check_every=5,
                        use_graph=False)
    # The two runs are the same kernels on the same inputs, but the gridding pass sums with FP32 atomics
    # in no fixed order, and in the learned stage a last-bit difference can move a hidden activation
    # across a BF16 rounding boundary (a 2^-9 relative step for that pixel).  Measured on a GB300:
    # five learned iterations repeated on identical inputs differ in ~900 of 4096 pixels (1.2e-7 rel.
    # L2), and repeated identical fallback runs differ from one another by up to 6e-5 (1.2e-4 seen
    # once against the two-stage run).  One BF16 step still separates this from every wrong restart
    # (the iterate doubles per learned iteration, so restarting one check late is 32x off).
    assert rel_l2(xg, to_host(xb)) <= 2.0 ** -8
