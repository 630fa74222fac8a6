"""FP64 oracle of the measurement operator Phi = G F Z (Eq. 1) and its adjoint.

Conventions (readings where the paper is silent):

* The image x is n x n, real, indexed x[a, b].  Pixel (a, b) sits at the
  centred offset p = (a - n/2, b - n/2); offset (0, 0) is the phase centre.
* Visibility m has angular frequencies omega[m] = (omega_0, omega_1) in
  rad/pixel; omega_0 pairs with image axis 0 and omega_1 with axis 1.
  The exact model is  y_m = sum_p x_p exp(-i omega.p) W_m(p)  with the
  w-modulation W_m(p) = exp(-2 pi i w_m (sqrt(1 - l^2 - m^2) - 1)),
  l = p_0 dl, m = p_1 dl (Eq. 1 with the w-effect of App. E).
* Z zero-pads onto a K x K grid (pixel offset p at grid index p mod K) and
  divides by the separable grid correction c(p_0) c(p_1), the continuous
  Fourier transform of the interpolation kernel (Eq. 1, Fessler 2003).
* F is the unnormalised forward 2-D DFT (scipy's fft2), F^H its exact adjoint
  (K^2 * ifft2).
* G row m holds the Kaiser-Bessel (KB) kernel taps around
  kappa = omega K / (2 pi): per axis the J integers k with |kappa - k| < J/2
  (first tap floor(kappa - J/2) + 1), wrapped mod K, weight psi(kappa - k).
  The grid is stored row-major, column index (k0 mod K) * K + (k1 mod K).
* KB shape parameter: beta = pi sqrt((J/sigma)^2 (sigma - 1/2)^2 - 0.8)
  (Beatty et al. 2005) with sigma = K/n; the paper only cites Fessler 2003.

w-folded rows (App. E; the paper defers the w-kernel to Dabbech et al. 2017
and gives no formula).  Reading used here, under the paraxial approximation
W ~ exp(i pi a (p_0^2 + p_1^2)), a = w dl^2, which is separable per axis:

* the w-kernel is the K-point DFT  w_hat[d] = K^-1 sum_p exp(i pi a q(p)) exp(2 pi i d p / K)
  of the chirp with its phase "frozen" outside the image: q(p) = p^2 for
  |p| <= n/2 and a smooth (C^2) monotone continuation beyond, flat at
  |p| = K/2 (see ``chirp_phase_q``).  Since q = p^2 on every image pixel, the
  untruncated row reproduces the paraxial model exactly up to the KB error.
* the row of G is the KB kernel convolved with that w-kernel,
  g(t) = sum_d w_hat[d] psi(t + d), restricted to the J_m x J_m taps nearest
  kappa (J_m = 7, 9, 12 or 16 by |w| quartile).  For w = 0 it is the KB row.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft
import scipy.sparse as sps
import scipy.special as spec

FFT_WORKERS = os.cpu_count() or 1   # threads of the FFT (the sparse products are single-threaded)


# ---------------------------------------------------------------- KB kernel
def kb_beta(J: int, sigma: float) -> float:
    """KB shape parameter for support J at oversampling sigma = K/n (Beatty et al. 2005)."""
    return float(np.pi * np.sqrt((J / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8))


def kb_psi(t, J: int, beta: float):
    """KB interpolation kernel psi(t) = I0(beta sqrt(1 - (2t/J)^2)) on |t| <= J/2, else 0."""
    t = np.asarray(t, dtype=np.float64)
    z = 1.0 - (2.0 * t / J) ** 2
    return np.where(z >= 0.0, spec.i0(beta * np.sqrt(np.maximum(z, 0.0))), 0.0)


def kb_correction(p, J: int, beta: float, K: int):
    """Grid correction c(p): continuous Fourier transform of psi at p/K cycles per cell.

    c(p) = J sinh(sqrt(beta^2 - s^2)) / sqrt(beta^2 - s^2), s = pi J p / K
    (the sin form when s > beta).
    """
    s = np.pi * J * np.asarray(p, dtype=np.float64) / K
    r2 = beta * beta - s * s
    out = np.empty_like(s)
    pos = r2 > 0
    r = np.sqrt(np.abs(r2))
    out[pos] = J * np.sinh(r[pos]) / r[pos]
    neg = r2 < 0
    out[neg] = J * np.sin(r[neg]) / r[neg]
    out[r2 == 0] = J
    return out


def pixel_offsets(n: int) -> np.ndarray:
    """Centred pixel offsets p = a - n/2 for a = 0..n-1."""
    return np.arange(n) - n // 2


def tap_start(kappa, J: int):
    """First of the J integers k with |kappa - k| < J/2: floor(kappa - J/2) + 1."""
    return np.floor(np.asarray(kappa) - J / 2.0).astype(np.int64) + 1


# ---------------------------------------------------------------- Z and F
class GridSpec:
    """Sizes and grid-correction table of one operator (n-pixel image, K-cell grid, KB J)."""

    def __init__(self, n: int, K: int, J: int = 7, beta: float | None = None):
        self.n, self.K, self.J = int(n), int(K), int(J)
        self.beta = kb_beta(J, K / n) if beta is None else float(beta)
        self.p = pixel_offsets(n)
        self.c = kb_correction(self.p, J, self.beta, K)


def zero_pad(gs: GridSpec, x: np.ndarray) -> np.ndarray:
    """Z: n x n image -> K x K grid, divided by c(p0) c(p1) (Eq. 1)."""
    grid = np.zeros((gs.K, gs.K), dtype=np.complex128)
    idx = gs.p % gs.K
    grid[np.ix_(idx, idx)] = x / np.outer(gs.c, gs.c)
    return grid


def zero_pad_adjoint(gs: GridSpec, grid: np.ndarray) -> np.ndarray:
    """Z^H: pick the image cells of the K x K grid and divide by c(p0) c(p1)."""
    idx = gs.p % gs.K
    return grid[np.ix_(idx, idx)] / np.outer(gs.c, gs.c)


def dft2(grid: np.ndarray) -> np.ndarray:
    """F: unnormalised forward 2-D DFT (scipy's FFT on all host cores)."""
    return sfft.fft2(grid, workers=FFT_WORKERS)


def dft2_adjoint(grid: np.ndarray) -> np.ndarray:
    """F^H: exact adjoint of the unnormalised DFT, K^2 ifft2."""
    return sfft.ifft2(grid, workers=FFT_WORKERS) * (grid.shape[0] * grid.shape[1])


# ---------------------------------------------------------------- w-kernel
def chirp_phase_q(p, n: int, K: int):
    """Phase profile q(p) of the frozen chirp: p^2 on the image, C^2 flat continuation.

    For h = n/2 < |p| <= K/2, with u = (|p| - h)/(K/2 - h):
      q = h^2 + n (K/2 - h) (u + u^2/2 - u^4 + 2 u^5 / 5),
    whose derivative n s(u), s(u) = 1 + u - 4u^3 + 2u^4, matches 2p and the
    zero second derivative at |p| = h and vanishes (with zero second
    derivative) at |p| = K/2, so the periodic profile is C^2.
    """
    a = np.abs(np.asarray(p, dtype=np.float64))
    h = n / 2.0
    out = a * a
    m = a > h
    u = (a[m] - h) / (K / 2.0 - h)
    out[m] = h * h + n * (K / 2.0 - h) * (u + u * u / 2.0 - u ** 4 + 2.0 * u ** 5 / 5.0)
    return out


def w_kernel(a, d, n: int, K: int) -> np.ndarray:
    """w_hat[m, j] = K^-1 sum_{p=-K/2}^{K/2-1} exp(i pi a_m q(p)) exp(2 pi i d_j p / K).

    Direct K-term sums (the definition), for each row parameter a_m = w_m dl^2.
    """
    a = np.atleast_1d(np.asarray(a, dtype=np.float64))
    d = np.asarray(d, dtype=np.float64)
    pk = np.arange(-K // 2, K // 2, dtype=np.float64)
    q = chirp_phase_q(pk, n, K)
    E = np.exp(2j * np.pi * np.outer(pk, d) / K) / K
    out = np.empty((a.size, d.size), dtype=np.complex128)
    for s in range(0, a.size, 256):
        out[s:s + 256] = np.exp(1j * np.pi * np.outer(a[s:s + 256], q)) @ E
    return out


def row_axis_weights(kappa, a, Jm: int, gs: GridSpec, w_hat_cache=None):
    """Per-axis weights of rows with support Jm: (taps k (R, Jm), g(kappa - k) (R, Jm)).

    g(t) = sum_d w_hat[d] psi(t + d) over all d with |t + d| <= J/2 (App. E
    reading above); with a = 0 this is psi itself.
    """
    kappa = np.asarray(kappa, dtype=np.float64)
    k = tap_start(kappa, Jm)[:, None] + np.arange(Jm)[None, :]
    t = kappa[:, None] - k
    a = np.asarray(a, dtype=np.float64)
    if np.all(a == 0.0):
        return k, kb_psi(t, gs.J, gs.beta).astype(np.complex128)
    D = int(np.ceil(Jm / 2.0 + gs.J / 2.0)) + 1
    dd = np.arange(-D, D + 1)
    what = w_kernel(a, dd, gs.n, gs.K) if w_hat_cache is None else w_hat_cache
    g = np.zeros(t.shape, dtype=np.complex128)
    for j, d in enumerate(dd):
        g += what[:, j:j + 1] * kb_psi(t + d, gs.J, gs.beta)
    return k, g


def degridding_matrix(gs: GridSpec, omega: np.ndarray, w=None, dl: float = 0.0,
                      J_per_row=None, rows=None, row_scale=None) -> sps.csr_matrix:
    """G as a scipy CSR matrix (len(rows) x K^2, complex128), rows in the given order.

    Row m: outer product of the two per-axis weight vectors of
    ``row_axis_weights`` (KB row, or the w-folded row when w and dl are set),
    times the data weight d_m when ``row_scale`` is given (Sec. 3: weighted
    data; the fidelity 1/2 ||D (G F Z x - y)||^2 with d_m = sqrt of the imaging
    weight makes Re{Phi^H Phi} delta the weighted dirty beam).
    """
    K = gs.K
    omega = np.asarray(omega, dtype=np.float64)
    m_all = omega.shape[0]
    rows = np.arange(m_all) if rows is None else np.asarray(rows)
    R = rows.size
    kap = omega[rows] * (K / (2.0 * np.pi))
    Jr = (np.full(R, gs.J, dtype=np.int64) if J_per_row is None
          else np.asarray(J_per_row, dtype=np.int64)[rows])
    a = (np.zeros(R) if (w is None or dl == 0.0)
         else np.asarray(w, dtype=np.float64)[rows] * dl * dl)
    nnz_row = Jr * Jr
    indptr = np.zeros(R + 1, dtype=np.int64)
    np.cumsum(nnz_row, out=indptr[1:])
    data = np.empty(indptr[-1], dtype=np.complex128)
    cols = np.empty(indptr[-1], dtype=np.int64)
    for Jm in np.unique(Jr):
        sel = np.nonzero(Jr == Jm)[0]
        for s in range(0, sel.size, 20000):
            ss = sel[s:s + 20000]
            k0, g0 = row_axis_weights(kap[ss, 0], a[ss], int(Jm), gs)
            k1, g1 = row_axis_weights(kap[ss, 1], a[ss], int(Jm), gs)
            wv = (g0[:, :, None] * g1[:, None, :]).reshape(ss.size, -1)
            cv = ((k0 % K)[:, :, None] * K + (k1 % K)[:, None, :]).reshape(ss.size, -1)
            pos = indptr[ss][:, None] + np.arange(Jm * Jm)[None, :]
            data[pos] = wv
            cols[pos] = cv
    if row_scale is not None:
        data *= np.repeat(np.asarray(row_scale, dtype=np.float64)[rows], nnz_row)
    return sps.csr_matrix((data, cols, indptr), shape=(R, K * K))


# ---------------------------------------------------------------- Phi
class Operator:
    """Phi = G F Z and its adjoints for one problem (FP64)."""

    def __init__(self, n: int, K: int, omega, w=None, dl: float = 0.0, J_per_row=None,
                 J: int = 7, beta: float | None = None, rows=None, row_scale=None):
        self.gs = GridSpec(n, K, J, beta)
        self.n, self.K = n, K
        self.G = degridding_matrix(self.gs, omega, w, dl, J_per_row, rows, row_scale)
        self.GH = self.G.conj().T.tocsr()
        self.M = self.G.shape[0]

    def forward(self, x) -> np.ndarray:
        """y = Phi x = G F Z x (Eq. 1).  x may be real or complex."""
        return self.G @ dft2(zero_pad(self.gs, x)).ravel()

    def adjoint_complex(self, r) -> np.ndarray:
        """Phi^H r = Z^H F^H G^H r (complex image)."""
        grid = (self.GH @ r).reshape(self.K, self.K)
        return zero_pad_adjoint(self.gs, dft2_adjoint(grid))

    def adjoint(self, r) -> np.ndarray:
        """Re{Phi^H r}, the real-image adjoint used by the gradient (App. A)."""
        return self.adjoint_complex(r).real

    def normal(self, x) -> np.ndarray:
        """Re{Phi^H Phi} x."""
        return self.adjoint(self.forward(x))


# ---------------------------------------------------------------- ground truth
def nudft(omega, x, w=None, dl: float = 0.0, paraxial: bool = True) -> np.ndarray:
    """Direct non-uniform DFT y_m = sum_p x_p exp(-i omega_m . p) W_m(p) (Eq. 1), O(M n^2).

    ``paraxial`` uses W = exp(i pi w dl^2 (p0^2 + p1^2)); otherwise the exact
    exp(-2 pi i w (sqrt(1 - l^2 - m^2) - 1)).
    """
    omega = np.asarray(omega, dtype=np.float64)
    n = x.shape[0]
    p = pixel_offsets(n).astype(np.float64)
    E0 = np.exp(-1j * omega[:, 0:1] * p[None, :])
    E1 = np.exp(-1j * omega[:, 1:2] * p[None, :])
    if w is None or dl == 0.0:
        return np.einsum("ma,ab,mb->m", E0, x, E1)
    w = np.asarray(w, dtype=np.float64)
    if paraxial:
        ch = np.exp(1j * np.pi * (w * dl * dl)[:, None] * (p * p)[None, :])
        return np.einsum("ma,ab,mb->m", E0 * ch, x, E1 * ch)
    l2 = ((p * dl) ** 2)[:, None] + ((p * dl) ** 2)[None, :]
    nm1 = np.sqrt(1.0 - l2) - 1.0
    out = np.empty(omega.shape[0], dtype=np.complex128)
    for m in range(omega.shape[0]):
        W = np.exp(-2j * np.pi * w[m] * nm1)
        out[m] = np.sum(np.outer(E0[m], E1[m]) * W * x)
    return out


def nudft_adjoint(omega, y, n: int) -> np.ndarray:
    """Direct adjoint of ``nudft`` without w: x_p = sum_m exp(+i omega_m . p) y_m (complex n x n)."""
    omega = np.asarray(omega, dtype=np.float64)
    p = pixel_offsets(n).astype(np.float64)
    E0 = np.exp(1j * omega[:, 0:1] * p[None, :])
    E1 = np.exp(1j * omega[:, 1:2] * p[None, :])
    return np.einsum("ma,m,mb->ab", E0, y, E1)
