"""FP64 oracle of uSARA's handcrafted denoiser (App. B): the SARA dictionary, the prox of the
weighted-l1 + positivity surrogate by sub-iterations, and the reweighted PnP-FB loop.

Test infrastructure: only the tests and the benchmark's CPU baseline use this module; the library
never does.

Readings (the paper names the model, not its implementation details):

* Psi is the normalised concatenation of P = 9 orthonormal bases, the Dirac basis and the 2-D
  Daubechies wavelet bases with 1..8 vanishing moments, each a 4-level separable DWT with periodic
  extension (so every basis is exactly orthonormal and Psi Psi^T = I: a tight frame):
      Psi^T x = [B_1 x, ..., B_9 x] / 3,   Psi c = sum_b B_b^T c_b / 3.
* The Daubechies low-pass filters come from the spectral factorisation of
  |m0(w)|^2 = cos^(2N)(w/2) P_N(sin^2(w/2)), P_N(y) = sum_{k<N} C(N-1+k, k) y^k, keeping the
  roots inside the unit circle (minimum phase), normalised to sum sqrt(2); the high-pass filter is
  g[k] = (-1)^k h[L-1-k].
* The log-sum prior lambda sum rho log(1 + |(Psi^T x)_n| / rho) is majorised at the current image by
  a weighted l1 norm with weights w_n = rho / (rho + |(Psi^T x)_n|) (its derivative at |u|); each
  convex surrogate is solved by FB with the prox of gamma lambda ||W Psi^T .||_1 + iota_+.
* That prox has no closed form; it is computed by dual forward-backward: with the Moreau identity
  the dual step of the weighted l1 term is a clip to [-t_n, t_n], t_n = gamma lambda w_n, so
      x_k = max(0, z - Psi u_k),   u_{k+1} = clip(u_k + mu Psi^T x_k, -t, t),   mu = 1 (||Psi|| = 1),
  stopped on the relative change of x.
* gamma lambda = tau / sqrt(2L) (Eq. lambda) and rho = gamma lambda.
"""
from __future__ import annotations

from math import comb

import numpy as np

LEVELS = 4
N_BASES = 9


# ---------------------------------------------------------------- Daubechies filters
def daubechies(N: int) -> np.ndarray:
    """Low-pass filter (length 2N) of the orthonormal Daubechies wavelet with N vanishing moments."""
    if N == 1:
        return np.array([1.0, 1.0]) / np.sqrt(2.0)
    # Q(z) = z^(N-1) P_N(y) with y = (2 - z - 1/z) / 4, i.e. y z = (-z^2 + 2 z - 1) / 4
    yz = np.array([-1.0, 2.0, -1.0]) / 4.0           # polynomial coefficients, highest power first
    Q = np.zeros(2 * N - 1)
    for k in range(N):
        term = np.array([1.0])
        for _ in range(k):
            term = np.polymul(term, yz)
        term = np.polymul(term, np.eye(1, N - k, 0).ravel())   # times z^(N-1-k)
        Q[-term.size:] += comb(N - 1 + k, k) * term
    roots = np.roots(Q)
    dQ = np.polyder(Q)
    for _ in range(3):  # Newton polish: the companion-matrix roots of degree 14 carry ~1e-12 errors
        roots = roots - np.polyval(Q, roots) / np.polyval(dQ, roots)
    inside = roots[np.abs(roots) < 1.0]
    Lz = np.real(np.poly(inside))
    h = np.array([1.0])
    for _ in range(N):
        h = np.polymul(h, np.array([1.0, 1.0]))
    h = np.real(np.polymul(h, Lz))
    return h * (np.sqrt(2.0) / h.sum())


def highpass(h: np.ndarray) -> np.ndarray:
    L = h.size
    return np.array([(-1) ** k * h[L - 1 - k] for k in range(L)])


# ---------------------------------------------------------------- periodic DWT
def _analysis_1d(x, f, axis):
    """a[i] = sum_k f[k] x[(2 i + k) mod n] along ``axis``."""
    out = 0.0
    for k, fk in enumerate(f):
        out = out + fk * np.take(np.roll(x, -k, axis=axis), np.arange(0, x.shape[axis], 2), axis=axis)
    return out


def _synthesis_1d(a, f, axis, n):
    """Adjoint of _analysis_1d: x[(2 i + k) mod n] += f[k] a[i]."""
    shape = list(a.shape)
    shape[axis] = n
    up = np.zeros(shape)
    idx = [slice(None)] * len(shape)
    idx[axis] = slice(0, n, 2)
    up[tuple(idx)] = a
    out = np.zeros(shape)
    for k, fk in enumerate(f):
        out = out + fk * np.roll(up, k, axis=axis)
    return out


def dwt2(x: np.ndarray, h: np.ndarray, levels: int = LEVELS) -> np.ndarray:
    """Orthonormal multi-level 2-D DWT with periodic extension, coefficients in one n x n array
    (approximation in the top-left corner of each level, details around it)."""
    g = highpass(h)
    c = np.array(x, dtype=np.float64)
    m = c.shape[0]
    for _ in range(levels):
        blk = c[:m, :m]
        lo = _analysis_1d(blk, h, 0)
        hi = _analysis_1d(blk, g, 0)
        ll, lh = _analysis_1d(lo, h, 1), _analysis_1d(lo, g, 1)
        hl, hh = _analysis_1d(hi, h, 1), _analysis_1d(hi, g, 1)
        c[:m, :m] = np.block([[ll, lh], [hl, hh]])
        m //= 2
    return c


def idwt2(c: np.ndarray, h: np.ndarray, levels: int = LEVELS) -> np.ndarray:
    """Inverse (= adjoint) of dwt2."""
    g = highpass(h)
    x = np.array(c, dtype=np.float64)
    m = x.shape[0] >> (levels - 1)
    for _ in range(levels):
        half = m // 2
        ll, lh = x[:half, :half], x[:half, half:m]
        hl, hh = x[half:m, :half], x[half:m, half:m]
        lo = _synthesis_1d(ll, h, 1, m) + _synthesis_1d(lh, g, 1, m)
        hi = _synthesis_1d(hl, h, 1, m) + _synthesis_1d(hh, g, 1, m)
        x[:m, :m] = _synthesis_1d(lo, h, 0, m) + _synthesis_1d(hi, g, 0, m)
        m *= 2
    return x


# ---------------------------------------------------------------- SARA dictionary
class Sara:
    """Psi^T and Psi of the normalised concatenation of the Dirac and db1..db8 bases."""

    def __init__(self, levels: int = LEVELS, bases=None):
        self.levels = levels
        self.filters = [daubechies(N) for N in range(1, 9)]
        self.bases = list(range(N_BASES)) if bases is None else list(bases)   # 0: Dirac, b: db_b
        self.scale = 1.0 / np.sqrt(len(self.bases))

    def analysis(self, x: np.ndarray) -> np.ndarray:
        """Psi^T x: (number of bases, n, n)."""
        out = []
        for b in self.bases:
            out.append(np.array(x, dtype=np.float64) if b == 0 else dwt2(x, self.filters[b - 1], self.levels))
        return np.stack(out) * self.scale

    def synthesis(self, c: np.ndarray) -> np.ndarray:
        """Psi c for c of shape (number of bases, n, n)."""
        x = 0.0
        for i, b in enumerate(self.bases):
            x = x + (c[i] if b == 0 else idwt2(c[i], self.filters[b - 1], self.levels))
        return x * self.scale


# ---------------------------------------------------------------- prox and loop
def reweighting_weights(coeffs: np.ndarray, rho: float) -> np.ndarray:
    """w_n = rho / (rho + |u_n|): the slope of rho log(1 + |u| / rho) at the current coefficients."""
    return rho / (rho + np.abs(coeffs))


def prox_weighted_l1_pos(psi: Sara, z: np.ndarray, t: np.ndarray, max_iter: int = 500, tol: float = 1e-8,
                         mu: float = 1.0, u0=None):
    """argmin_x 1/2 ||x - z||^2 + sum_n t_n |(Psi^T x)_n| + iota_+(x) by dual forward-backward.
    Returns (x, u, iterations)."""
    u = np.zeros((len(psi.bases),) + z.shape) if u0 is None else np.array(u0, dtype=np.float64)
    x = np.maximum(0.0, z - psi.synthesis(u))
    it = 0
    for it in range(1, max_iter + 1):
        u = np.clip(u + mu * psi.analysis(x), -t, t)
        x_new = np.maximum(0.0, z - psi.synthesis(u))
        change = np.linalg.norm(x_new - x) / max(np.linalg.norm(x_new), 1e-300)
        x = x_new
        if change < tol:
            break
    return x, u, it


def usara(op, y, gamma: float, gamma_lambda: float, rho: float, n_reweights: int, fb_iters: int,
          prox_iters: int = 100, psi: Sara | None = None, x0=None, prox_tol: float = 1e-6):
    """Reweighted PnP-FB with the SARA prior: n_reweights + 1 convex surrogates of fb_iters FB
    iterations each (the dual variable of the prox is warm-started from one call to the next)."""
    psi = Sara() if psi is None else psi
    n = op.n
    x = np.zeros((n, n)) if x0 is None else np.array(x0, dtype=np.float64)
    w = np.ones((len(psi.bases), n, n))
    u = None
    for _ in range(n_reweights + 1):
        for _ in range(fb_iters):
            z = x - gamma * op.adjoint(op.forward(x) - y)
            x, u, _ = prox_weighted_l1_pos(psi, z, gamma_lambda * w, prox_iters, prox_tol, u0=u)
        w = reweighting_weights(psi.analysis(x), rho)
    return x
