"""Pins of the uSARA oracle (App. B): Daubechies filters, periodic DWT, SARA tight frame, the
weighted-l1 + positivity prox and the reweighting weights."""
import numpy as np
import pytest

from oracle import fb as ofb
from oracle import sara as osa


@pytest.mark.parametrize("N", range(1, 9))
def test_daubechies_filters_are_orthonormal_with_n_vanishing_moments(N):
    h = osa.daubechies(N)
    assert h.size == 2 * N
    assert h.sum() == pytest.approx(np.sqrt(2.0), abs=1e-12)
    for m in range(N):                                   # sum h_k h_{k+2m} = delta_m
        assert np.dot(h[:h.size - 2 * m], h[2 * m:]) == pytest.approx(1.0 if m == 0 else 0.0, abs=1e-10)
    g = osa.highpass(h)
    k = np.arange(h.size)
    for p in range(N):                                   # the wavelet kills polynomials of degree < N
        assert abs(np.dot(g, k.astype(float) ** p)) <= 1e-8 * max(1.0, float(np.abs(k ** p).max()))


def test_db2_closed_form():
    s3 = np.sqrt(3.0)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * np.sqrt(2.0))
    h = osa.daubechies(2)
    assert np.allclose(h, ref, atol=1e-12) or np.allclose(h, ref[::-1], atol=1e-12)


def test_dwt_is_orthonormal_and_invertible():
    x = np.random.default_rng(1).standard_normal((32, 32))
    for N in (1, 3, 8):
        h = osa.daubechies(N)
        c = osa.dwt2(x, h)
        assert np.linalg.norm(c) == pytest.approx(np.linalg.norm(x), rel=1e-12)
        assert np.allclose(osa.idwt2(c, h), x, atol=1e-11)


def test_db1_one_level_is_the_2x2_haar_block_transform():
    x = np.random.default_rng(2).standard_normal((8, 8))
    c = osa.dwt2(x, osa.daubechies(1), levels=1)
    a, hh, vv, d = ofb.haar_analysis(x)                  # the FB oracle's one-level Haar on 2 x 2 blocks
    assert np.allclose(c[:4, :4], a, atol=1e-12)
    assert np.allclose(np.abs(c[4:, 4:]), np.abs(d), atol=1e-12)
    assert np.allclose(np.sort(np.abs(np.concatenate([c[:4, 4:].ravel(), c[4:, :4].ravel()]))),
                       np.sort(np.abs(np.concatenate([hh.ravel(), vv.ravel()]))), atol=1e-12)


def test_sara_is_a_tight_frame():
    psi = osa.Sara()
    x = np.random.default_rng(3).standard_normal((32, 32))
    c = psi.analysis(x)
    assert c.shape == (9, 32, 32)
    assert np.linalg.norm(c) == pytest.approx(np.linalg.norm(x), rel=1e-12)
    assert np.allclose(psi.synthesis(c), x, atol=1e-11)
    r = np.random.default_rng(4).standard_normal(c.shape)   # adjoint pair
    assert np.sum(psi.analysis(x) * r) == pytest.approx(np.sum(x * psi.synthesis(r)), rel=1e-12)


def test_prox_special_cases():
    z = np.random.default_rng(5).standard_normal((16, 16))
    psi = osa.Sara(levels=2)
    x, _, _ = osa.prox_weighted_l1_pos(psi, z, np.zeros((9, 16, 16)), 50)
    assert np.allclose(x, np.maximum(z, 0), atol=1e-12)            # no penalty: the projection
    dirac = osa.Sara(levels=2, bases=[0])
    t = 0.3
    x, _, _ = osa.prox_weighted_l1_pos(dirac, z, np.full((1, 16, 16), t), 2000, 1e-12)
    assert np.allclose(x, np.maximum(z - t, 0), atol=1e-8)          # identity dictionary: closed form


def test_prox_minimises_its_objective():
    rng = np.random.default_rng(6)
    z = rng.standard_normal((16, 16)) + 0.5
    psi = osa.Sara(levels=2)
    t = 0.05 * (1 + rng.random((9, 16, 16)))
    x, _, it = osa.prox_weighted_l1_pos(psi, z, t, 1500, 1e-10)

    def obj(v):
        return 0.5 * np.sum((v - z) ** 2) + np.sum(t * np.abs(psi.analysis(v)))
    assert np.all(x >= 0)
    base = obj(x)
    for _ in range(30):
        v = np.maximum(0.0, x + 1e-3 * rng.standard_normal(x.shape))
        assert obj(v) >= base - 1e-9


def test_reweighting_weights_are_the_log_sum_slope():
    rho = 0.2
    u = np.linspace(-2, 2, 41)
    u = u[np.abs(u) > 1e-3]
    f = lambda v: rho * np.log1p(np.abs(v) / rho)
    e = 1e-6
    slope = (f(np.abs(u) + e) - f(np.abs(u) - e)) / (2 * e)
    assert np.allclose(osa.reweighting_weights(u, rho), slope, rtol=1e-8)


def test_usara_with_the_dirac_basis_alone_is_fb_with_soft_threshold_and_positivity():
    from oracle import nufft as nu
    rng = np.random.default_rng(7)
    n, K, M = 16, 32, 300
    op = nu.Operator(n, K, rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (M, 2)))
    x_true = np.maximum(rng.standard_normal((n, n)), 0)
    y = op.forward(x_true) + 0.01 * (rng.standard_normal(M) + 1j * rng.standard_normal(M))
    L, _, _ = ofb.power_iteration(op, rng.standard_normal((n, n)), 1000, 1e-10)
    gamma, t = ofb.step_size(L), 1e-2
    x = osa.usara(op, y, gamma, t, t, 0, 20, prox_iters=3000, psi=osa.Sara(levels=2, bases=[0]))
    x_ref, _ = ofb.pnp_fb(op, y, gamma, lambda z: np.maximum(z - t, 0.0), 20)
    assert np.allclose(x, x_ref, atol=1e-7 * np.abs(x_ref).max())


def test_reweighting_sharpens_the_sparsity():
    from oracle import nufft as nu
    rng = np.random.default_rng(8)
    n, K, M = 16, 32, 400
    op = nu.Operator(n, K, rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (M, 2)))
    x_true = np.zeros((n, n))
    x_true[rng.integers(0, n, 6), rng.integers(0, n, 6)] = 1.0
    y = op.forward(x_true) + 0.01 * (rng.standard_normal(M) + 1j * rng.standard_normal(M))
    L, _, _ = ofb.power_iteration(op, rng.standard_normal((n, n)), 1000, 1e-10)
    gamma, t = ofb.step_size(L), 2e-2
    psi = osa.Sara(levels=2)
    x0 = osa.usara(op, y, gamma, t, t, 0, 10, prox_iters=30, psi=psi)
    x2 = osa.usara(op, y, gamma, t, t, 1, 10, prox_iters=30, psi=psi)
    # the log-sum prior favours fewer, larger coefficients than its l1 surrogate at the same threshold
    small0 = np.sum(np.abs(psi.analysis(x0)) > 1e-3)
    small2 = np.sum(np.abs(psi.analysis(x2)) > 1e-3)
    assert small2 <= small0
    assert ofb.snr_db(x_true, x2) >= ofb.snr_db(x_true, x0) - 0.5
