"""FP64 oracle of the forward-backward (FB) iteration and its parameters (App. A, B, F).

Readings where the paper is silent:

* The plain (handcrafted) denoiser is the one-level orthonormal 2-D Haar
  transform on 2 x 2 blocks, soft-thresholding all four subbands (the
  regulariser sums over every dictionary coefficient, App. B), synthesis,
  then projection on the positive orthant, in that order.  For orthonormal
  Haar the first three steps are the exact prox of t ||Psi^T .||_1; the
  composition with positivity is a one-shot approximation of the joint prox,
  which has no closed form (App. B).
* x^0 = 0; the stopping test ||x^{k+1} - x^k|| / ||x^{k+1}|| < tol is applied
  only when tol > 0.
* Power iteration starts from a caller-supplied vector and stops when the
  relative change of the estimate falls below tol.
* Complex noise of "standard deviation tau" (Eq. 1) means E|n|^2 = tau^2.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- data fidelity
def data_fidelity(op, x, y) -> float:
    """f(x) = 1/2 ||Phi x - y||_2^2 (App. A)."""
    r = op.forward(x) - y
    return 0.5 * float(np.vdot(r, r).real)


def gradient(op, x, y) -> np.ndarray:
    """grad f(x) = Re{Phi^H (Phi x - y)} (App. A)."""
    return op.adjoint(op.forward(x) - y)


def gradient_step(op, x, y, gamma: float) -> np.ndarray:
    """Forward step z = x - gamma grad f(x) (Eq. fb)."""
    return x - gamma * gradient(op, x, y)


def power_iteration(op, v0, max_it: int = 1000, tol: float = 1e-10):
    """L = ||Re{Phi^H Phi}||_S by power iteration (App. A: L is the Lipschitz constant).

    Returns (L, v, iterations).
    """
    v = np.asarray(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    L = 0.0
    it = 0
    for it in range(1, max_it + 1):
        u = op.normal(v)
        L_new = float(np.linalg.norm(u))
        v = u / L_new
        if it > 1 and abs(L_new - L) <= tol * L_new:
            L = L_new
            break
        L = L_new
    return L, v, it


def step_size(L: float, factor: float = 1.98) -> float:
    """gamma = 1.98 / L (App. B), inside the convergence range gamma < 2/L (Eq. fb)."""
    return factor / L


def psf_peak(op) -> float:
    """beta = max_i (Re{Phi^H Phi} delta)_i, delta = 1 at the phase centre (App. F footnote)."""
    n = op.n
    d = np.zeros((n, n))
    d[n // 2, n // 2] = 1.0
    return float(op.normal(d).max())


# ---------------------------------------------------------------- parameters
def noise_level_image(tau: float, L: float) -> float:
    """Image-domain noise estimate tau / sqrt(2L) (Eq. lambda, App. B)."""
    return tau / np.sqrt(2.0 * L)


def soft_threshold_from_noise(tau: float, L: float) -> float:
    """gamma*lambda = tau / sqrt(2L) (Eq. lambda); also rho = gamma*lambda (App. B)."""
    return noise_level_image(tau, L)


def dirty_peak(op, y, beta: float) -> float:
    """Peak of the normalised dirty image max(Re{Phi^H y}) / beta (App. F)."""
    return float(op.adjoint(y).max() / beta)


def dynamic_range(peak: float, noise_level: float) -> float:
    """Target dynamic range = peak / (tau / sqrt(2L)) (App. F)."""
    return peak / noise_level


def sigma_from_dynamic_range(dr: float) -> float:
    """Training noise level of a denoiser trained for dynamic range dr: sigma = 1/dr (App. F)."""
    return 1.0 / dr


def sigma_heuristic(tau: float, alpha: float, L: float) -> float:
    """sigma = tau / (alpha sqrt(2L)) (Eq. sigma)."""
    return tau / (alpha * np.sqrt(2.0 * L))


def alpha_for_denoiser(tau: float, L: float, sigma_train: float) -> float:
    """Rescaling alpha that matches data to a fixed denoiser: solves Eq. sigma for alpha (App. C, F)."""
    return tau / (sigma_train * np.sqrt(2.0 * L))


# ---------------------------------------------------------------- Haar prox
def haar_analysis(x: np.ndarray):
    """One-level orthonormal 2-D Haar on 2 x 2 blocks -> (approx, h, v, d) subbands."""
    x00, x01 = x[0::2, 0::2], x[0::2, 1::2]
    x10, x11 = x[1::2, 0::2], x[1::2, 1::2]
    a = 0.5 * (x00 + x01 + x10 + x11)
    h = 0.5 * (x00 - x01 + x10 - x11)
    v = 0.5 * (x00 + x01 - x10 - x11)
    d = 0.5 * (x00 - x01 - x10 + x11)
    return a, h, v, d


def haar_synthesis(a, h, v, d) -> np.ndarray:
    """Inverse of ``haar_analysis`` (its transpose)."""
    n0, n1 = a.shape
    x = np.empty((2 * n0, 2 * n1), dtype=np.result_type(a, np.float64))
    x[0::2, 0::2] = 0.5 * (a + h + v + d)
    x[0::2, 1::2] = 0.5 * (a - h + v - d)
    x[1::2, 0::2] = 0.5 * (a + h - v - d)
    x[1::2, 1::2] = 0.5 * (a - h - v + d)
    return x


def soft_threshold(c, t: float):
    """prox of t|.|: sign(c) max(|c| - t, 0) (App. A); zero at the tie |c| = t."""
    return np.sign(c) * np.maximum(np.abs(c) - t, 0.0)


def haar_denoise(z: np.ndarray, t: float, positivity: bool = True) -> np.ndarray:
    """Plain denoiser: Haar analysis, soft-threshold all subbands, synthesis, positivity."""
    out = haar_synthesis(*(soft_threshold(c, t) for c in haar_analysis(z)))
    return np.maximum(out, 0.0) if positivity else out


# ---------------------------------------------------------------- FB loop
def pnp_fb(op, y, gamma: float, denoiser, iters: int, x0=None, tol: float = 0.0,
           x_true=None, alpha: float = 1.0):
    """x^{k+1} = D(x^k - gamma grad f(x^k)) (Eq. fb with a plug-in denoiser D).

    With ``alpha`` the loop solves the rescaled problem of App. C (Eq. invpb2),
    y / alpha = Phi (x / alpha) + n / alpha: it starts from x0 / alpha, iterates
    on y / alpha, and the returned image is alpha times its result (the SNR in
    the history is that of alpha x).
    Returns (x, history) where history holds per iteration the relative change
    ||x^{k+1} - x^k|| / ||x^{k+1}||, f(x^{k+1}) and, if x_true is given, the SNR.
    """
    n = op.n
    x = np.zeros((n, n)) if x0 is None else np.array(x0, dtype=np.float64) / alpha
    y = np.asarray(y) / alpha
    hist = {"rel_change": [], "f": [], "snr": []}
    for _ in range(iters):
        x_new = denoiser(gradient_step(op, x, y, gamma))
        nx = np.linalg.norm(x_new)
        rc = np.linalg.norm(x_new - x) / nx if nx > 0 else 0.0
        x = x_new
        hist["rel_change"].append(rc)
        hist["f"].append(data_fidelity(op, x, y))
        if x_true is not None:
            hist["snr"].append(snr_db(x_true, alpha * x))
        if tol > 0 and rc < tol:
            break
    return alpha * x, hist


def snr_db(x_true, x) -> float:
    """Reconstruction SNR 20 log10(||x_true|| / ||x_true - x||); the paper gives no definition."""
    return float(20.0 * np.log10(np.linalg.norm(x_true) / np.linalg.norm(x_true - x)))
