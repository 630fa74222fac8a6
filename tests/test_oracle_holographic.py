"""Pins of the holographic normal-operator oracle (App. E, Eq. phidagphi)."""
import numpy as np

import synth
from oracle import fb as ofb
from oracle import holographic as oh
from oracle import nufft as nu


def _op(seed=0, n=16, K=32, M=400, w=True):
    rng = np.random.default_rng(4000 + seed)
    omega = rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (M, 2))
    if not w:
        return nu.Operator(n, K, omega), rng
    ww = rng.uniform(-1.0, 1.0, M)
    return nu.Operator(n, K, omega, ww, np.sqrt(4.0 / (n * K)), synth.j_per_row_by_w_quartile(ww)), rng


def test_holographic_matrix_is_hermitian_and_banded():
    op, _ = _op()
    H = oh.holographic_matrix(op)
    assert abs(H - H.conj().T).max() <= 1e-12 * abs(H).max()
    K = op.K
    r, c = H.nonzero()
    dr = (r // K - c // K + K // 2) % K - K // 2
    dc = (r % K - c % K + K // 2) % K - K // 2
    assert np.abs(dr).max() <= 15 and np.abs(dc).max() <= 15      # |k - k'| < J_max = 16 per axis


def test_holographic_normal_and_gradient_equal_the_plain_ones():
    for w in (False, True):
        op, rng = _op(1, w=w)
        H = oh.holographic_matrix(op)
        x = rng.standard_normal((op.n, op.n))
        y = rng.standard_normal(op.M) + 1j * rng.standard_normal(op.M)
        ref = op.normal(x)
        assert np.linalg.norm(oh.normal(op, H, x) - ref) <= 1e-12 * np.linalg.norm(ref)
        g = oh.gradient(op, H, oh.dirty_grid(op, y), x)
        g_ref = ofb.gradient(op, x, y)
        assert np.linalg.norm(g - g_ref) <= 1e-12 * np.linalg.norm(g_ref)


def test_holographic_matrix_entries_are_sums_over_rows():
    # H[k, k'] = sum_m conj(G_mk) G_mk', checked entry by entry on a few pairs
    op, _ = _op(2, M=60, w=False)
    H = oh.holographic_matrix(op).toarray()
    G = op.G.toarray()
    rng = np.random.default_rng(5)
    for _ in range(20):
        m = rng.integers(op.M)
        ks = np.nonzero(G[m])[0]
        k, k2 = rng.choice(ks, 2)
        assert abs(H[k, k2] - np.sum(np.conj(G[:, k]) * G[:, k2])) <= 1e-12 * abs(H).max()
