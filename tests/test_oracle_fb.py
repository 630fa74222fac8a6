"""Pins of the FP64 forward-backward oracle (App. A, B, F of arXiv 2207.11336)."""
import os

import numpy as np
import pytest

import synth
from oracle import fb
from oracle import nufft as nu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "appF_parameters.txt")


def _small_problem(n=8, K=16, M=300, seed=11):
    rng = np.random.default_rng(seed)
    omega = rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (M, 2))
    return nu.Operator(n, K, omega), rng


def _dense_normal(op):
    n = op.n
    A = np.empty((n * n, n * n))
    for i in range(n * n):
        e = np.zeros(n * n)
        e[i] = 1.0
        A[:, i] = op.normal(e.reshape(n, n)).ravel()
    return A


def test_gradient_matches_finite_differences():
    op, rng = _small_problem()
    x = rng.random((op.n, op.n))
    y = op.forward(rng.random((op.n, op.n))) + 0.01 * synth.complex_normal(op.M, rng)
    g = fb.gradient(op, x, y)
    h = 1e-5
    for _ in range(6):
        i, j = rng.integers(0, op.n, 2)
        e = np.zeros_like(x)
        e[i, j] = h
        fd = (fb.data_fidelity(op, x + e, y) - fb.data_fidelity(op, x - e, y)) / (2 * h)
        assert g[i, j] == pytest.approx(fd, rel=1e-7, abs=1e-9 * abs(g).max())


def test_normal_operator_is_symmetric_psd():
    op, _ = _small_problem()
    A = _dense_normal(op)
    assert np.allclose(A, A.T, atol=1e-9 * abs(A).max())
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > -1e-9 * abs(A).max()


def test_power_iteration_equals_dense_spectral_norm():
    op, rng = _small_problem()
    A = _dense_normal(op)
    lam = np.linalg.eigvalsh(0.5 * (A + A.T)).max()
    L, v, it = fb.power_iteration(op, rng.standard_normal((op.n, op.n)), 5000, 1e-14)
    assert L == pytest.approx(lam, rel=1e-10)


def test_psf_peak_equals_M_and_bounds_L():
    # unit weights: (Re{Phi^H Phi} delta)(0) = sum_m |1|^2 = M up to NUFFT error
    op, rng = _small_problem(n=16, K=32, M=400)
    beta = fb.psf_peak(op)
    assert beta == pytest.approx(op.M, rel=1e-5)
    L, _, _ = fb.power_iteration(op, rng.standard_normal((16, 16)), 3000, 1e-12)
    assert L >= beta * (1 - 1e-9)


def test_appF_printed_parameter_arithmetic():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for band, noise_mjy, peak_jy, dr_printed in rows[:2]:
        dr = fb.dynamic_range(float(peak_jy), float(noise_mjy) * 1e-3)
        # printed with two significant figures ("5x10^5" for 4.93e5)
        assert dr == pytest.approx(float(dr_printed), rel=0.02), band
    _, dr_train, sigma = rows[2]
    assert fb.sigma_from_dynamic_range(float(dr_train)) == pytest.approx(float(sigma), rel=1e-12)
    # Eq. sigma and its inverse agree
    tau, L = 0.3, 7.0e4
    a = fb.alpha_for_denoiser(tau, L, 2.5e-6)
    assert fb.sigma_heuristic(tau, a, L) == pytest.approx(2.5e-6, rel=1e-12)
    assert fb.soft_threshold_from_noise(tau, L) == pytest.approx(tau / np.sqrt(2 * L))


def test_haar_is_orthonormal():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((8, 12))
    c = fb.haar_analysis(x)
    assert np.allclose(fb.haar_synthesis(*c), x, atol=1e-15)
    assert sum(np.sum(ci ** 2) for ci in c) == pytest.approx(np.sum(x ** 2), rel=1e-14)
    # explicit 4x4 analysis matrix is orthogonal
    B = np.array([fb.np.concatenate([ci.ravel() for ci in fb.haar_analysis(e.reshape(2, 2))])
                  for e in np.eye(4)])
    assert np.allclose(B @ B.T, np.eye(4), atol=1e-15)


@pytest.mark.parametrize("c,t", [(1.0, 0.5), (0.2, 0.5), (0.25, 0.5), (3.0, 0.0), (-1.0, 0.3)])
def test_haar_denoise_constant_block_closed_form(c, t):
    z = np.full((2, 2), c)
    expect = max(0.0, c - t / 2) if 2 * c > t else 0.0
    if c < 0:
        expect = 0.0
    assert np.allclose(fb.haar_denoise(z, t), expect, atol=1e-15)


def test_haar_denoise_t0_is_positivity():
    z = np.random.default_rng(4).standard_normal((6, 6))
    assert np.allclose(fb.haar_denoise(z, 0.0), np.maximum(z, 0.0), atol=1e-15)


def test_haar_soft_threshold_is_prox():
    # u* = Psi S_t Psi^T z minimises t||Psi^T u||_1 + 1/2||z - u||^2 (App. A prox)
    rng = np.random.default_rng(5)
    z = rng.standard_normal((4, 4))
    t = 0.4
    u = fb.haar_denoise(z, t, positivity=False)

    def obj(v):
        return t * sum(np.abs(ci).sum() for ci in fb.haar_analysis(v)) + 0.5 * np.sum((z - v) ** 2)
    base = obj(u)
    for _ in range(300):
        assert obj(u + 1e-3 * rng.standard_normal(u.shape)) >= base - 1e-12


@pytest.mark.parametrize("mode", ["positivity", "haar"])
def test_fb_objective_monotone_with_exact_prox(mode):
    # Exact prox + gamma < 2/L => F(x^{k+1}) <= F(x^k) (sufficient decrease of FB).
    op, rng = _small_problem(n=16, K=32, M=600)
    x_true = np.maximum(rng.standard_normal((16, 16)), 0)
    y = op.forward(x_true) + 0.05 * synth.complex_normal(op.M, rng)
    L, _, _ = fb.power_iteration(op, rng.standard_normal((16, 16)), 3000, 1e-12)
    gamma = fb.step_size(L)
    t = 0.0 if mode == "positivity" else 0.05 * np.sqrt(op.M)
    lam = t / gamma
    if mode == "positivity":
        den = lambda z: np.maximum(z, 0.0)           # noqa: E731
        reg = lambda v: 0.0                          # noqa: E731
    else:
        den = lambda z: fb.haar_denoise(z, t, positivity=False)   # noqa: E731
        reg = lambda v: lam * sum(np.abs(c).sum() for c in fb.haar_analysis(v))  # noqa: E731
    x = np.zeros((16, 16))
    F = [fb.data_fidelity(op, x, y) + reg(x)]
    for _ in range(40):
        x = den(fb.gradient_step(op, x, y, gamma))
        F.append(fb.data_fidelity(op, x, y) + reg(x))
    assert all(b <= a * (1 + 1e-12) + 1e-12 for a, b in zip(F, F[1:]))
    assert F[-1] < F[0]


def test_pnp_fb_fixed_point_and_history():
    op, rng = _small_problem(n=16, K=32, M=600)
    x_true = np.maximum(rng.standard_normal((16, 16)), 0)
    y = op.forward(x_true)
    L, _, _ = fb.power_iteration(op, rng.standard_normal((16, 16)), 3000, 1e-12)
    gamma = fb.step_size(L)
    den = lambda z: np.maximum(z, 0.0)   # noqa: E731
    x, h = fb.pnp_fb(op, y, gamma, den, 3000, tol=1e-12, x_true=x_true)
    assert np.allclose(den(fb.gradient_step(op, x, y, gamma)), x, atol=1e-8 * abs(x).max())
    assert len(h["rel_change"]) == len(h["f"]) == len(h["snr"])


def test_weighted_operator_dirty_beam_and_adjoint():
    """Data weights d_m on the rows (Sec. 3, Briggs): the weighted dirty beam at the phase centre is
    sum_m d_m^2 (y_m = 1 exactly for a delta at the centre, so only the NUFFT error remains), which
    fails if the weights were applied once or not squared; the adjoint identity holds to 1e-12."""
    rng = np.random.default_rng(21)
    n, K, M = 16, 32, 500
    omega = rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (M, 2))
    d = np.sqrt(synth.briggs_weights(omega, n, 0.0))
    op = nu.Operator(n, K, omega, J=7, row_scale=d)
    delta = np.zeros((n, n))
    delta[n // 2, n // 2] = 1.0
    assert fb.psf_peak(op) == pytest.approx(np.sum(d ** 2), rel=2e-6)
    assert np.allclose(op.forward(delta), d, rtol=0, atol=2e-6)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    r = synth.complex_normal(M, rng)
    lhs = np.vdot(op.forward(x), r)
    rhs = np.vdot(x, op.adjoint_complex(r))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(op.forward(x)) * np.linalg.norm(r)


def test_alpha_rescaling_is_exact_for_the_haar_loop():
    """App. C, Eq. invpb2: soft thresholding and positivity are positively homogeneous, so the loop on
    y / alpha with threshold t / alpha, multiplied by alpha, is the loop on y with threshold t."""
    op, rng = _small_problem(n=16, K=32, M=800, seed=3)
    x_true = np.maximum(rng.standard_normal((16, 16)), 0)
    y = op.forward(x_true) + 0.05 * synth.complex_normal(op.M, rng)
    L, _, _ = fb.power_iteration(op, rng.standard_normal((16, 16)), 2000, 1e-12)
    gamma, t, alpha = fb.step_size(L), 0.02, 7.5
    x1, _ = fb.pnp_fb(op, y, gamma, lambda z: fb.haar_denoise(z, t), 40)
    x2, _ = fb.pnp_fb(op, y, gamma, lambda z: fb.haar_denoise(z, t / alpha), 40, alpha=alpha)
    assert np.allclose(x1, x2, rtol=1e-12, atol=1e-12 * abs(x1).max())
    x3, _ = fb.pnp_fb(op, y, gamma, lambda z: fb.haar_denoise(z, t), 40, alpha=alpha)
    assert not np.allclose(x1, x3, rtol=1e-6)   # the threshold does not scale by itself


def test_snr_db_closed_forms():
    """SNR = 20 log10(||x|| / ||x - x_hat||) on cases with a closed form: x_hat = (1 - e) x gives
    -20 log10(e) (20 dB at e = 0.1; an SNR taken against x_hat instead of x would give 19.08), a
    perturbation orthogonal to x of relative norm 10^(-k/20) gives k dB, x_hat = 0 gives 0 dB, and
    the value is invariant to a common scale (a swapped ratio would give negative values)."""
    rng = np.random.default_rng(31)
    x = rng.standard_normal((12, 12))
    for e in (0.1, 0.01, 0.5):
        assert fb.snr_db(x, (1.0 - e) * x) == pytest.approx(-20.0 * np.log10(e), rel=1e-12)
    p = rng.standard_normal(x.shape)
    p -= np.vdot(x, p) / np.vdot(x, x) * x                     # orthogonal to x
    for k in (3.0, 17.5, 40.0):
        xh = x + p * (np.linalg.norm(x) / np.linalg.norm(p)) * 10.0 ** (-k / 20.0)
        assert fb.snr_db(x, xh) == pytest.approx(k, abs=1e-10)
        assert fb.snr_db(3.7 * x, 3.7 * xh) == pytest.approx(k, abs=1e-10)
    assert fb.snr_db(x, np.zeros_like(x)) == pytest.approx(0.0, abs=1e-12)


def _dense_real_system(op, y):
    """Phi as a dense complex matrix (columns Phi e_i), stacked as the real least-squares system
    [Re Phi; Im Phi] x = [Re y; Im y] of 1/2 ||Phi x - y||^2 over real images x."""
    n = op.n
    cols = []
    for i in range(n * n):
        e = np.zeros(n * n)
        e[i] = 1.0
        cols.append(op.forward(e.reshape(n, n)))
    P = np.stack(cols, axis=1)
    return np.vstack([P.real, P.imag]), np.concatenate([y.real, y.imag])


@pytest.mark.parametrize("den", ["identity", "positivity"])
def test_pnp_fb_converges_to_the_library_least_squares_solution(den):
    """Eq. fb with D = identity is gradient descent on 1/2 ||Phi x - y||^2 and with D = positivity
    projected gradient descent: run to convergence, the oracle's loop must reach the minimiser that
    numpy's lstsq, respectively scipy's NNLS, computes from the dense system (a wrong sign, a dropped
    y term or a conjugated operand in the gradient converges elsewhere or diverges)."""
    from scipy.optimize import nnls
    op, rng = _small_problem(n=6, K=12, M=200, seed=41)
    x_true = rng.standard_normal((6, 6))
    y = op.forward(x_true) + 0.3 * synth.complex_normal(op.M, rng)
    A, b = _dense_real_system(op, y)
    if den == "identity":
        ref = np.linalg.lstsq(A, b, rcond=None)[0].reshape(6, 6)
        D = lambda z: z                      # noqa: E731
    else:
        ref = nnls(A, b, maxiter=10000)[0].reshape(6, 6)
        D = lambda z: np.maximum(z, 0.0)     # noqa: E731
    L = np.linalg.norm(A, 2) ** 2
    x, _ = fb.pnp_fb(op, y, fb.step_size(L), D, 20000, tol=1e-15)
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
