"""Pins of the Jacobian oracle of the CNN denoiser (firm non-expansiveness measure, Eq. training_loss)."""
import numpy as np
import pytest

import synth
from oracle import cnn as ocnn
from oracle import jacobian as oj


def _net(seed, channels=4, depth=3, scale=1.0):
    return synth.cnn_init(np.random.default_rng(seed), channels=channels, depth=depth, last_scale=scale)


def _img(seed, n=10):
    return np.random.default_rng(seed).standard_normal((n, n))


def test_jvp_matches_central_differences():
    params, z, v = _net(1), _img(2), _img(3)
    h = 1e-6
    fd = (ocnn.network(params, z + h * v) - ocnn.network(params, z - h * v)) / (2 * h)
    j = oj.jvp(params, z, v)
    assert np.linalg.norm(j - fd) <= 1e-6 * np.linalg.norm(fd)


def test_vjp_is_the_adjoint_of_jvp():
    params, z = _net(4, depth=4), _img(5, 12)
    v, w = _img(6, 12), _img(7, 12)
    lhs = float(np.sum(oj.jvp(params, z, v) * w))
    rhs = float(np.sum(v * oj.vjp(params, z, w)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_power_iteration_equals_dense_svd():
    # dense Jacobian by central differences of the network (independent of jvp/vjp)
    params, z = _net(8), _img(9, 8)
    n = z.size
    h = 1e-6
    J = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        J[:, k] = ((ocnn.network(params, z + e.reshape(z.shape)) -
                    ocnn.network(params, z - e.reshape(z.shape))) / (2 * h)).ravel()
    s_ref = np.linalg.svd(np.eye(n) - 2 * J, compute_uv=False)[0]
    s, v = oj.q_jacobian_norm(params, z, _img(10, 8), 400)
    assert s == pytest.approx(s_ref, rel=1e-6)
    assert np.linalg.norm(v) == pytest.approx(1.0)


def test_constant_network_gives_unit_norm():
    # zero last layer: N is constant, J_N = 0 and J_Q = I
    params = _net(11)
    params[-1] = (np.zeros_like(params[-1][0]), params[-1][1])
    s, _ = oj.q_jacobian_norm(params, _img(12), _img(13), 3)
    assert s == pytest.approx(1.0, abs=1e-15)


def test_bf16_mirror_differs_by_rounding_only():
    # with the same ReLU masks the BF16 mirror differs from FP64 by its roundings (weights and
    # 3 stored tangents, each <= 2^-9 relative); the masks themselves may flip between a BF16 and
    # an FP64 forward pass, where the Jacobian jumps, so they are shared here
    params, z, v = _net(14, channels=8, depth=4), _img(15, 16), _img(16, 16)
    _, acts = ocnn.network(params, z, bf16=True, keep=True)
    a, b = oj.jvp(params, z, v, bf16=True, acts=acts), oj.jvp(params, z, v, acts=acts)
    assert np.linalg.norm(a - b) <= 2.0 ** -6 * np.linalg.norm(b)


def test_penalty_gradient_matches_central_differences():
    params = _net(17, channels=4, depth=3)
    z = np.stack([_img(18), _img(19)])
    v = np.stack([_img(20), _img(21)])
    v /= np.linalg.norm(v, axis=(1, 2), keepdims=True)
    lam, eps = 0.7, 0.5
    P, grads, n2 = oj.fne_penalty_and_grads(params, z, v, lam, eps)
    assert P == pytest.approx(lam / 2 * sum(max(a, 1 - eps) for a in n2))
    h = 1e-6
    for li, idx in [(0, (1, 0, 2, 1)), (1, (2, 3, 0, 0)), (2, (0, 1, 1, 2))]:
        def pen(delta):
            p2 = [(W.copy(), b.copy()) for W, b in params]
            p2[li][0][idx] += delta
            return oj.fne_penalty_and_grads(p2, z, v, lam, eps)[0]
        fd = (pen(h) - pen(-h)) / (2 * h)
        assert grads[li][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    assert all(np.all(db == 0) for _, db in grads)


def test_penalty_inactive_below_the_bound():
    params = _net(22)
    z, v = _img(23)[None], _img(24)[None]
    v = v / np.linalg.norm(v)
    P, grads, n2 = oj.fne_penalty_and_grads(params, z, v, 1.0, 1.0 - 2 * n2_of(params, z, v))
    assert all(np.all(dW == 0) for dW, _ in grads)


def n2_of(params, z, v):
    return oj.fne_penalty_and_grads(params, z, v, 1.0, 0.0)[2][0]
