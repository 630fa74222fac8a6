"""GPU Jacobian of the CNN denoiser vs the oracle: ||grad (2D - I)||_S by power iteration
(the firm non-expansiveness measure of Eq. training_loss, App. C).

Both sides freeze the ReLU masks of their own BF16 forward pass and store tangents and
back-propagated gradients in BF16 (the oracle mirrors the rounding points, sums in FP64; the GPU
sums in FP32 on the tensor cores).  A mask can differ where a pre-activation sits within rounding
of zero, and the Jacobian jumps there, so the bounds are a few BF16 units rather than one.
"""
import os

import numpy as np
import pytest

import synth
from oracle import jacobian as oj

from gpu_common import pnp, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _inputs(B, s, seed, sigma=0.05):
    rng = np.random.default_rng(seed)
    u = np.stack([synth.training_image(s, rng) for _ in range(B)])
    z = (u + sigma * rng.standard_normal((B, s, s))).astype(np.float32)
    v0 = rng.standard_normal((B, s, s)).astype(np.float32)
    return z, v0


@pytest.mark.parametrize("iters", [1, 8])
def test_jacobian_norm_matches_oracle(iters):
    B, s = 2, 24
    params = synth.cnn_init(np.random.default_rng(31), 64, 8, last_scale=1.0)
    z, v0 = _inputs(B, s, 32)
    tr = pnp.CnnTrainer(params, B, s)
    sig, v = tr.jacobian_norm(torch.from_numpy(z).cuda(), torch.from_numpy(v0).cuda(), iters)
    v = v.cpu().numpy().astype(np.float64)
    for b in range(B):
        s_ref, v_ref = oj.q_jacobian_norm(params, z[b].astype(np.float64), v0[b].astype(np.float64), iters,
                                          bf16=True)
        assert sig[b] == pytest.approx(s_ref, rel=2.0 ** -6)
        cos = float(np.vdot(v[b], v_ref) / (np.linalg.norm(v[b]) * np.linalg.norm(v_ref)))
        assert cos >= 0.99
        assert np.linalg.norm(v[b]) == pytest.approx(1.0, rel=1e-5)
    tr.close()


def test_constant_network_has_unit_jacobian_norm():
    B, s = 2, 16
    params = synth.cnn_init(np.random.default_rng(33), 64, 8, last_scale=1.0)
    params[-1] = (np.zeros_like(params[-1][0]), params[-1][1])      # N constant: J_Q = I
    z, v0 = _inputs(B, s, 34)
    tr = pnp.CnnTrainer(params, B, s)
    sig, _ = tr.jacobian_norm(torch.from_numpy(z).cuda(), torch.from_numpy(v0).cuda(), 3)
    assert np.allclose(sig, 1.0, rtol=0, atol=1e-6)
    tr.close()


def test_trained_denoiser_jacobian_norm_is_reported():
    """The committed network (trained without the penalty) at its training noise level."""
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2207_11336_gb300", "weights", "dncnn_C3.npz")
    if not os.path.exists(path):
        pytest.skip("no trained weights")
    from paper_2207_11336_gb300.train_denoiser import load
    params, meta = load(path)
    sigma = float(meta["sigma"])
    B, s = 4, 128
    rng = np.random.default_rng(35)
    u = np.stack([synth.training_image(s, rng) for _ in range(B)])
    z = (u + sigma * rng.standard_normal((B, s, s))).astype(np.float32)
    v0 = rng.standard_normal((B, s, s)).astype(np.float32)
    tr = pnp.CnnTrainer(params, B, s)
    sig, _ = tr.jacobian_norm(torch.from_numpy(z).cuda(), torch.from_numpy(v0).cuda(), 30)
    print("||grad(2D - I)||_S of the trained network at sigma = %.3g:" % sigma, sig)
    assert np.all(np.isfinite(sig)) and np.all(sig > 0.5)
    tr.close()


def test_penalty_gradients_match_oracle():
    """The penalty's weight gradients (trainer gradients with the penalty minus without it) against
    the oracle's back-propagation through the frozen-mask tangent network; iters = 0 fixes v."""
    B, s, sigma = 2, 24, 0.05
    params = synth.cnn_init(np.random.default_rng(41), 64, 8, last_scale=0.3)
    rng = np.random.default_rng(42)
    u = np.stack([synth.training_image(s, rng) for _ in range(B)]).astype(np.float32)
    nz = rng.standard_normal((B, s, s)).astype(np.float32)
    v0 = rng.standard_normal((B, s, s)).astype(np.float32)
    tr = pnp.CnnTrainer(params, B, s)
    ud, nd, vd = (torch.from_numpy(a).cuda() for a in (u, nz, v0))
    tr.step(ud, nd, sigma, update=False)
    _, g1 = tr.read(weights=False, grads=True, clear_grads=True)
    loss, pen = tr.step_fne(ud, nd, sigma, vd, 0, lam=1.0, eps=1.0, update=False, want_values=True)
    _, g2 = tr.read(weights=False, grads=True, clear_grads=True)
    tr.close()
    gp = pnp.unpack_cnn_weights(g2.astype(np.float64) - g1.astype(np.float64))
    z = (u + np.float32(sigma) * nz).astype(np.float64)
    v = v0.astype(np.float64) / np.linalg.norm(v0.astype(np.float64), axis=(1, 2), keepdims=True)
    P, grads, _ = oj.fne_penalty_and_grads(params, z, v, 1.0, 1.0, bf16=True)
    assert pen == pytest.approx(P, rel=2.0 ** -6)
    for li, ((dW, _), (gW, gb)) in enumerate(zip(grads, gp)):
        cos = float(np.vdot(gW, dW) / (np.linalg.norm(gW) * np.linalg.norm(dW)))
        assert cos >= 0.995, (li, cos)
        # the gradient reaching layer 1 has passed 7 BF16 tangents and 7 BF16 back-propagated
        # gradients, and its sums cancel: a few percent of its norm, not one BF16 unit
        assert np.linalg.norm(gW - dW) <= 2.0 ** -4 * np.linalg.norm(dW), li
        assert np.abs(gb).max() <= 1e-3 * max(np.abs(g1).max(), 1e-30)   # no bias gradient


def test_penalised_training_lowers_the_jacobian_norm():
    B, s = 4, 32
    params = synth.cnn_init(np.random.default_rng(43), 64, 8, last_scale=1.0)
    rng = np.random.default_rng(44)
    u = torch.from_numpy(np.stack([synth.training_image(s, rng) for _ in range(B)]).astype(np.float32)).cuda()
    gen = torch.Generator(device="cuda").manual_seed(45)
    tr = pnp.CnnTrainer(params, B, s, lr=2e-4)
    zt = u + 0.05 * torch.randn(u.shape, device="cuda", generator=gen)
    v0 = torch.randn(u.shape, device="cuda", generator=gen)
    before, _ = tr.jacobian_norm(zt.contiguous(), v0, 20)
    for _ in range(60):
        nz = torch.randn(u.shape, device="cuda", generator=gen)
        vv = torch.randn(u.shape, device="cuda", generator=gen)
        tr.step_fne(u, nz, 0.05, vv, 3, lam=1.0, eps=0.05)
    after, _ = tr.jacobian_norm(zt.contiguous(), v0, 20)
    tr.close()
    print("||grad(2D - I)||_S before / after 60 penalised steps:", before, after)
    assert after.max() < before.max()
