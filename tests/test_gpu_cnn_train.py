"""GPU training kernels of the CNN denoiser (App. C) vs the oracle's gradients.

The oracle back-propagates with the same BF16 rounding points (weights, hidden
activations, pre-activation gradients) and FP64 sums; its gradients are pinned
to finite differences in test_oracle_cnn.py.  The last layer starts near zero
so the l1 residual never sits at a sign change, where the two sides could
legitimately disagree.  The GPU sums in FP32 (tensor cores) and rounds the
back-propagated gradients to BF16; weight gradients are sums of terms of both
signs, so the bound is the standard one for floating-point sums: per layer,
||g_gpu - g_ref|| <= 2^-7 ||sum of |terms| ||; a cosine >= 0.999 with the
reference catches indexing errors.
"""
import numpy as np
import pytest

import synth
from oracle import cnn as ocnn

from gpu_common import pnp, require_gpu, torch

pytestmark = pytest.mark.gpu
BF16_U = 2.0 ** -8


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _batch(B, s, seed):
    rng = np.random.default_rng(seed)
    u = np.stack([synth.training_image(s, rng) for _ in range(B)]).astype(np.float32)
    nz = rng.standard_normal((B, s, s)).astype(np.float32)
    return u, nz


def test_gradients_match_oracle():
    B, s, sigma = 2, 32, 0.1
    params = synth.cnn_init(np.random.default_rng(11), 64, 8, last_scale=0.01)
    u, nz = _batch(B, s, 12)
    tr = pnp.CnnTrainer(params, B, s, lr=1e-4)
    loss = tr.step(torch.from_numpy(u).cuda(), torch.from_numpy(nz).cuda(), sigma, update=False, want_loss=True)
    _, g = tr.read(weights=False, grads=True)
    gp = pnp.unpack_cnn_weights(g)
    loss_ref, grads, absg = ocnn.l1_loss_and_grads(params, u[:, None].astype(np.float64),
                                                   nz[:, None].astype(np.float64), sigma, bf16=True,
                                                   with_abs=True)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    errs = []
    for li, ((dW, db), (aW, ab), (gW, gb)) in enumerate(zip(grads, absg, gp)):
        eW = np.linalg.norm(gW - dW) / np.linalg.norm(aW)
        eb = np.linalg.norm(gb - db) / max(np.linalg.norm(ab), 1e-30)
        cos = float(np.vdot(gW, dW) / (np.linalg.norm(gW) * np.linalg.norm(dW)))
        errs.append((li, float(eW), float(eb), cos))
    print("per-layer (layer, err W / |terms|, err b / |terms|, cosine):", errs)
    assert all(e[1] <= 2 * BF16_U and e[2] <= 2 * BF16_U and e[3] >= 0.999 for e in errs), errs


def test_training_reduces_loss():
    B, s, sigma = 4, 64, 0.05
    params = synth.cnn_init(np.random.default_rng(13), 64, 8, last_scale=0.1)
    tr = pnp.CnnTrainer(params, B, s, lr=5e-4)
    rng = np.random.default_rng(14)
    pool = [synth.training_image(s, rng).astype(np.float32) for _ in range(16)]
    losses = []
    for it in range(60):
        idx = rng.choice(len(pool), B)
        u = torch.from_numpy(np.stack([pool[i] for i in idx])).cuda()
        nz = torch.randn((B, s, s), device="cuda", generator=torch.Generator("cuda").manual_seed(it))
        losses.append(tr.step(u, nz, sigma, update=True, want_loss=True))
    assert np.mean(losses[-10:]) < 0.8 * np.mean(losses[:5])
    w, _ = tr.read()
    assert all(np.isfinite(W).all() and np.isfinite(b).all() for W, b in w)


def test_gpu_adam_matches_oracle_over_three_updates():
    """The GPU Adam kernel against the oracle's adam_step on the same gradients: each step the
    gradients the GPU accumulated are read back and the oracle applies its update to the weights it
    read before; the moments carry over three updates (bias correction at t = 1, 2, 3).  FP32 on
    the GPU against FP64: the weights agree to 1e-6 of the step size."""
    B, s, sigma, lr = 2, 32, 0.1, 1e-3
    params = synth.cnn_init(np.random.default_rng(21), 64, 8, last_scale=0.05)
    tr = pnp.CnnTrainer(params, B, s, lr=lr)
    st = ocnn.adam_init(params)
    w_prev, _ = tr.read()
    for step in range(3):
        u, nz = _batch(B, s, 30 + step)
        tr.step(torch.from_numpy(u).cuda(), torch.from_numpy(nz).cuda(), sigma, update=False)
        _, g = tr.read(weights=False, grads=True)
        tr.apply_update()
        w_gpu, _ = tr.read()
        ref = ocnn.adam_step(w_prev, pnp.unpack_cnn_weights(g), st, lr=lr)
        for (Wg, bg), (Wr, br) in zip(w_gpu, ref):
            assert np.abs(Wg - Wr).max() <= 1e-6 * lr + 1e-7 * np.abs(Wr).max(), step
            assert np.abs(bg - br).max() <= 1e-6 * lr + 1e-7 * np.abs(br).max(), step
        w_prev = w_gpu
