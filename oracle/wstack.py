"""FP64 oracle of the w-stacked measurement operator (App. E, Eq. phip and Eq. phidagphi).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module; the library never does.

The rows are split into P w-stacks.  Stack p has a centre w_p; its operator is
Phi_p = G_p F Z_p where

* Z_p multiplies the image by the stack's centre chirp before zero-padding:
  pixel p = (p0, p1) gets exp(i pi a_p (p0^2 + p1^2)), a_p = w_p dl^2 (the
  paraxial w-modulation of the plain operator in ``nufft``, evaluated at w_p;
  on image pixels the frozen-chirp profile q(p) equals p^2, so this factor is
  exact), then divides by the grid correction and pads (``nufft.zero_pad``);
* G_p holds the w-folded rows of ``nufft.degridding_matrix`` built with the
  residual w_m - w_p of each of its rows, so the row kernels carry only the
  offset chirp exp(i pi (a_m - a_p) q(p)).

Since exp(i pi a_m p^2) = exp(i pi a_p p^2) exp(i pi (a_m - a_p) p^2), the
untruncated stacked rows give the same operator as the untruncated plain rows;
truncated, the smaller residual chirp needs a smaller support J_m for the same
accuracy, which is the point of the hybrid.  Phi stacks the Phi_p row blocks
(Eq. phip) and Phi^H Phi = sum_p Phi_p^H Phi_p (Eq. phidagphi).
"""
from __future__ import annotations

import numpy as np

from . import nufft as nu


def centre_chirp(n: int, w_centre: float, dl: float) -> np.ndarray:
    """The image modulation of Z_p: exp(i pi a_p (p0^2 + p1^2)), a_p = w_p dl^2, on the n x n pixels."""
    p = nu.pixel_offsets(n).astype(np.float64)
    ch = np.exp(1j * np.pi * w_centre * dl * dl * p * p)
    return np.outer(ch, ch)


def forward_rows(n: int, K: int, omega, w, dl: float, stack, w_centres, J_per_row, x, rows) -> np.ndarray:
    """Rows ``rows`` of Phi x for the stacked operator, one full-size FFT per stack they touch."""
    rows = np.asarray(rows)
    stack = np.asarray(stack)
    w_res = np.asarray(w, dtype=np.float64) - np.asarray(w_centres, dtype=np.float64)[stack]
    gs = nu.GridSpec(n, K)
    out = np.zeros(rows.size, dtype=np.complex128)
    for s in np.unique(stack[rows]):
        sel = np.nonzero(stack[rows] == s)[0]
        Xhat = nu.dft2(nu.zero_pad(gs, x * centre_chirp(n, float(w_centres[s]), dl))).ravel()
        G = nu.degridding_matrix(gs, omega, w_res, dl, J_per_row, rows[sel])
        out[sel] = G @ Xhat
    return out


class StackedOperator:
    """Phi = [Phi_1; ...; Phi_P] with Phi_p = G_p F Z_p (FP64); rows keep the caller's order."""

    def __init__(self, n: int, K: int, omega, w, dl: float, stack, w_centres, J_per_row=None,
                 J: int = 7, beta: float | None = None):
        omega = np.asarray(omega, dtype=np.float64)
        w = np.asarray(w, dtype=np.float64)
        stack = np.asarray(stack, dtype=np.int64)
        self.w_centres = np.asarray(w_centres, dtype=np.float64)
        self.n, self.K, self.M = n, K, omega.shape[0]
        self.P = self.w_centres.size
        Jr = None if J_per_row is None else np.asarray(J_per_row, dtype=np.int64)
        self.rows, self.ops, self.chirps = [], [], []
        for s in range(self.P):
            r = np.nonzero(stack == s)[0]
            self.rows.append(r)
            self.ops.append(nu.Operator(n, K, omega[r], w[r] - self.w_centres[s], dl,
                                        None if Jr is None else Jr[r], J, beta))
            self.chirps.append(centre_chirp(n, self.w_centres[s], dl))

    def forward(self, x) -> np.ndarray:
        """y = Phi x: row block p is G_p F Z_p x (Eq. phip)."""
        y = np.zeros(self.M, dtype=np.complex128)
        for r, op, C in zip(self.rows, self.ops, self.chirps):
            if r.size:
                y[r] = op.forward(x * C)
        return y

    def adjoint_complex(self, r) -> np.ndarray:
        """Phi^H r = sum_p Z_p^H F^H G_p^H r_p (complex image)."""
        out = np.zeros((self.n, self.n), dtype=np.complex128)
        for rows, op, C in zip(self.rows, self.ops, self.chirps):
            if rows.size:
                out += np.conj(C) * op.adjoint_complex(np.asarray(r)[rows])
        return out

    def adjoint(self, r) -> np.ndarray:
        """Re{Phi^H r}, the real-image adjoint of the gradient step."""
        return self.adjoint_complex(r).real

    def normal(self, x) -> np.ndarray:
        """Re{Phi^H Phi} x = Re sum_p Phi_p^H Phi_p x (Eq. phidagphi)."""
        return self.adjoint(self.forward(x))
