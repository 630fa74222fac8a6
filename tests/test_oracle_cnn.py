"""Pins of the FP64 CNN oracle (App. C, D of arXiv 2207.11336)."""
import numpy as np
import pytest
from scipy import signal

import synth
from oracle import cnn


def _tiny_net(rng, ch=4, depth=2):
    shapes = [(ch, 1)] + [(ch, ch)] * (depth - 2) + [(1, ch)]
    return [(rng.normal(0, 0.5, (co, ci, 3, 3)), rng.normal(0, 0.1, co)) for co, ci in shapes]


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 9, 7))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    out = cnn.conv_forward(x, W, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(signal.correlate2d(x[bi, c], W[o, c], mode="same") for c in range(3))
            assert np.allclose(out[bi, o], ref, atol=1e-12)


def test_col2im_is_adjoint_of_im2col():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 2, 5, 6))
    c = rng.standard_normal((1, 18, 30))
    assert np.vdot(cnn.im2col(x), c) == pytest.approx(np.vdot(x, cnn.col2im(c, x.shape)), rel=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    params = _tiny_net(rng, ch=4, depth=3)
    u = rng.random((2, 1, 16, 16))
    noise = rng.standard_normal(u.shape)
    loss, grads = cnn.l1_loss_and_grads(params, u, noise, 0.1)
    h = 1e-6
    for li in range(len(params)):
        for _ in range(3):
            W, b = params[li]
            idx = tuple(rng.integers(0, s) for s in W.shape)
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = [p if i != li else (Wp, b) for i, p in enumerate(params)]
            pm = [p if i != li else (Wm, b) for i, p in enumerate(params)]
            fd = (cnn.l1_loss_and_grads(pp, u, noise, 0.1)[0] -
                  cnn.l1_loss_and_grads(pm, u, noise, 0.1)[0]) / (2 * h)
            assert grads[li][0][idx] == pytest.approx(fd, rel=1e-6, abs=1e-10)
        j = rng.integers(0, len(b))
        bp, bm = b.copy(), b.copy()
        bp[j] += h
        bm[j] -= h
        fd = (cnn.l1_loss_and_grads([p if i != li else (W, bp) for i, p in enumerate(params)], u, noise, 0.1)[0]
              - cnn.l1_loss_and_grads([p if i != li else (W, bm) for i, p in enumerate(params)], u, noise, 0.1)[0]) / (2 * h)
        assert grads[li][1][j] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    v = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.uniform(-8, 3, 1000),
                        [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0]])
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.to_bf16(v), ref)


def test_faceted_equals_unfaceted():
    # App. D: a halo >= the receptive radius (8 px for 8 layers) makes faceting exact.
    rng = np.random.default_rng(5)
    params = synth.cnn_init(rng, channels=8, depth=8)
    z = rng.random((40, 36))
    full = cnn.denoise(params, z)
    fac = cnn.denoise_faceted(params, z, [13, 15, 12], [20, 16], halo=8)
    assert np.allclose(fac, full, atol=1e-13)
    small = cnn.denoise_faceted(params, z, [13, 15, 12], [20, 16], halo=4)
    assert not np.allclose(small, full, atol=1e-6)


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(6)
    params = _tiny_net(rng)
    grads = [(rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for W, b in params]
    st = cnn.adam_init(params)
    new = cnn.adam_step(params, grads, st, lr=1e-3)
    for (W, b), (W2, b2), (gW, gb) in zip(params, new, grads):
        assert np.allclose(W2 - W, -1e-3 * np.sign(gW), atol=1e-8)
        assert np.allclose(b2 - b, -1e-3 * np.sign(gb), atol=1e-8)


def test_residual_form_and_positivity():
    rng = np.random.default_rng(7)
    params = _tiny_net(rng)
    z = rng.standard_normal((10, 10))
    d = cnn.denoise(params, z, positivity=False)
    assert np.allclose(d, z - cnn.network(params, z))
    assert np.array_equal(cnn.denoise(params, z), np.maximum(d, 0))


def test_adam_matches_torch_over_several_steps():
    """The oracle's Adam beyond the first step (momentum and bias correction) against torch.optim.Adam
    fed the same gradients, an independent implementation of Kingma & Ba's update."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    params = _tiny_net(rng)
    st = cnn.adam_init(params)
    tp = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for W, b in params for a in (W, b)]
    opt = torch.optim.Adam(tp, lr=2e-3, betas=(0.9, 0.999), eps=1e-8)
    cur = params
    for step in range(5):
        grads = [(rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for W, b in params]
        cur = cnn.adam_step(cur, grads, st, lr=2e-3)
        for t, g in zip(tp, [a for gW, gb in grads for a in (gW, gb)]):
            t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        mine = [a for W, b in cur for a in (W, b)]
        for a, t in zip(mine, tp):
            assert np.allclose(a, t.detach().numpy(), rtol=1e-12, atol=1e-14), step
