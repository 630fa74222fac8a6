"""Pins of the FP64 measurement-operator oracle against things other than itself.

Each test checks the oracle with a library routine, a closed form, an
invariant or brute force (Eq. 1, App. A, App. E of arXiv 2207.11336).
"""
import numpy as np
import pytest
from scipy import integrate

import synth
from oracle import nufft as nu


def _rng(s=0):
    return np.random.default_rng(1000 + s)


def test_nudft_equals_fft_on_grid_frequencies():
    # omega = 2 pi j / n on the n-point DFT grid: the direct NUDFT with centred
    # pixels must equal (-1)^(j0+j1) fft2(x)[j] (library routine).
    n = 16
    rng = _rng(1)
    x = rng.random((n, n))
    j = rng.integers(-n // 2, n // 2, (40, 2))
    omega = 2 * np.pi * j / n
    y = nu.nudft(omega, x)
    ref = np.fft.fft2(x)[j[:, 0] % n, j[:, 1] % n] * (-1.0) ** (j[:, 0] + j[:, 1])
    assert np.allclose(y, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_exact_w_term_tends_to_paraxial():
    # exp(-2 pi i w (sqrt(1-r^2)-1)) = exp(i pi w r^2) (1 + O(w r^4)): the gap
    # must shrink like dl^4 (pins the sign and scale of both w forms).
    n = 16
    rng = _rng(2)
    x = rng.random((n, n))
    omega = rng.uniform(-2, 2, (30, 2))
    w = rng.uniform(-3e4, 3e4, 30)
    errs = []
    for dl in (2e-4, 1e-4):
        ye = nu.nudft(omega, x, w, dl, paraxial=False)
        yp = nu.nudft(omega, x, w, dl, paraxial=True)
        y0 = nu.nudft(omega, x)
        assert np.linalg.norm(yp - y0) > 10 * np.linalg.norm(ye - yp)
        errs.append(np.linalg.norm(ye - yp))
    assert 12 < errs[0] / errs[1] < 20          # ~2^4


@pytest.mark.parametrize("p", [0, 3, 17, 31, 32, 40])
def test_grid_correction_is_kernel_fourier_transform(p):
    J, K, n = 7, 64, 32
    beta = nu.kb_beta(J, K / n)
    val, _ = integrate.quad(lambda t: float(nu.kb_psi(t, J, beta)) * np.cos(2 * np.pi * t * p / K),
                            -J / 2, J / 2, epsabs=0, epsrel=1e-13, limit=200)
    assert nu.kb_correction(np.array([p]), J, beta, K)[0] == pytest.approx(val, rel=1e-11)


def test_kb_beta_value():
    # Beatty et al. 2005 at J = 7, sigma = 2.
    assert nu.kb_beta(7, 2.0) == pytest.approx(np.pi * np.sqrt(3.5 ** 2 * 1.5 ** 2 - 0.8))
    assert nu.kb_beta(7, 2.0) == pytest.approx(16.2522, abs=1e-4)


def test_tap_window_has_J_taps_within_half_support():
    kap = np.array([-3.2, 0.0, 0.5, 10.49, 10.5, 511.9])
    for J in (7, 8, 12):
        k = nu.tap_start(kap, J)[:, None] + np.arange(J)
        assert np.all(np.abs(kap[:, None] - k) <= J / 2)
        assert np.all(np.abs(kap - (nu.tap_start(kap, J) - 1)) >= J / 2)


def test_nufft_matches_direct_nudft_at_J7_sigma2():
    # spec accuracy pin: relative L2 <= 1e-6 at J = 7, 2x oversampling.
    n, K, M = 32, 64, 2000
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    x = prob["x_true"]
    op = nu.Operator(n, K, prob["omega"])
    y = op.forward(x)
    yd = nu.nudft(prob["omega"], x)
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) <= 1e-6


def test_operator_scale_point_source():
    # A unit point source at the phase centre gives y_m = 1 for every m.
    n, K = 16, 32
    rng = _rng(3)
    omega = rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (500, 2))
    d = np.zeros((n, n))
    d[n // 2, n // 2] = 1.0
    y = nu.Operator(n, K, omega).forward(d)
    assert np.max(np.abs(y - 1.0)) < 2e-6


def _w_problem(n=16, K=32, M=300, seed=4, supports=(7, 9, 12, 16)):
    rng = _rng(seed)
    omega = rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (M, 2))
    w = rng.uniform(-1.0, 1.0, M)
    dl = np.sqrt(4.0 / (n * K))            # largest |w| spreads 4 cells
    Jr = synth.j_per_row_by_w_quartile(w, supports)
    return omega, w, dl, Jr


@pytest.mark.parametrize("with_w", [False, True])
def test_adjoint_identity(with_w):
    n, K = 16, 32
    omega, w, dl, Jr = _w_problem(n, K)
    op = nu.Operator(n, K, omega, w if with_w else None, dl if with_w else 0.0,
                     Jr if with_w else None)
    rng = _rng(5)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    r = rng.standard_normal(op.M) + 1j * rng.standard_normal(op.M)
    lhs = np.vdot(r, op.forward(x))                 # <Phi x, r>
    rhs = np.vdot(op.adjoint_complex(r), x)         # <x, Phi^H r>
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(op.forward(x)) * np.linalg.norm(r)
    xr = x.real
    assert np.vdot(r, op.forward(xr)).real == pytest.approx(np.sum(xr * op.adjoint(r)), rel=1e-12)


def test_w_kernel_is_delta_at_zero_w_and_inverts():
    n, K = 16, 32
    d = np.arange(-K // 2, K // 2)
    wh0 = nu.w_kernel([0.0], d, n, K)[0]
    assert np.allclose(wh0, (d == 0).astype(float), atol=1e-15)
    a = 0.01
    wh = nu.w_kernel([a], d, n, K)[0]
    # inverse DFT (library routine) of w_hat over one period gives the chirp
    pk = np.arange(-K // 2, K // 2)
    chirp = np.array([np.sum(wh * np.exp(-2j * np.pi * d * p / K)) for p in pk])
    assert np.allclose(chirp, np.exp(1j * np.pi * a * nu.chirp_phase_q(pk, n, K)), atol=1e-13)
    # chirp phase profile is p^2 on the image, C^1 and flat at K/2
    q = nu.chirp_phase_q(np.arange(-n // 2, n // 2 + 1), n, K)
    assert np.allclose(q, np.arange(-n // 2, n // 2 + 1) ** 2)
    e = 1e-6
    dq = (nu.chirp_phase_q(np.array([K / 2]), n, K) - nu.chirp_phase_q(np.array([K / 2 - e]), n, K)) / e
    assert abs(dq[0]) < 1e-4
    h = n / 2
    dq_in = (nu.chirp_phase_q(np.array([h + e]), n, K) - nu.chirp_phase_q(np.array([h - e]), n, K)) / (2 * e)
    assert dq_in[0] == pytest.approx(2 * h, rel=1e-6)


def test_w_zero_rows_equal_kb_rows():
    n, K = 16, 32
    omega, w, dl, Jr = _w_problem(n, K)
    w0 = np.zeros_like(w)
    Gw = nu.degridding_matrix(nu.GridSpec(n, K), omega, w0 + 1e-300, dl, np.full_like(Jr, 7))
    Gk = nu.degridding_matrix(nu.GridSpec(n, K), omega)
    assert abs(Gw - Gk).max() <= 1e-12 * abs(Gk).max()


def test_untruncated_w_rows_reproduce_paraxial_nudft():
    # With J_m = K the folded row is the whole KB (x) w-kernel convolution, so
    # the operator equals the paraxial direct NUDFT up to the KB error.
    n, K, M = 16, 32, 120
    omega, w, dl, _ = _w_problem(n, K, M)
    x = _rng(6).random((n, n))
    op = nu.Operator(n, K, omega, w, dl, np.full(M, K, dtype=np.int64))
    y = op.forward(x)
    yd = nu.nudft(omega, x, w, dl, paraxial=True)
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < 5e-6


def test_w_rows_truncation_error_decreases_with_support():
    n, K, M = 16, 32, 200
    omega, w, dl, _ = _w_problem(n, K, M)
    x = _rng(7).random((n, n))
    yd = nu.nudft(omega, x, w, dl, paraxial=True)
    errs = []
    for J in (7, 9, 12, 16):
        y = nu.Operator(n, K, omega, w, dl, np.full(M, J, dtype=np.int64)).forward(x)
        errs.append(np.linalg.norm(y - yd) / np.linalg.norm(yd))
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-2


def test_nudft_adjoint_identity():
    n = 12
    rng = _rng(8)
    omega = rng.uniform(-np.pi, np.pi, (70, 2))
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    r = rng.standard_normal(70) + 1j * rng.standard_normal(70)
    lhs = np.vdot(r, nu.nudft(omega, x))
    rhs = np.vdot(nu.nudft_adjoint(omega, r, n), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
