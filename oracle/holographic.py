"""FP64 oracle of the holographic form of the normal operator (App. E, Eq. phidagphi).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU baseline use this
module; the library never does.

Phi^H Phi = Z^H F^H H F Z with the holographic matrix H = G^H G (N' x N', Hermitian): de-gridding
and gridding in one sparse operator that no longer depends on the number of data M.  The gradient
of the data term is then Re{Z^H F^H (H F Z x - G^H y)}: the dirty grid G^H y is formed once.
H couples grid cells k, k' only when some row of G touches both, so |k - k'| < J per axis.
"""
from __future__ import annotations

import numpy as np

from . import nufft as nu


def holographic_matrix(op: nu.Operator):
    """H = G^H G as a scipy CSR matrix (complex128)."""
    return (op.GH @ op.G).tocsr()


def dirty_grid(op: nu.Operator, y) -> np.ndarray:
    """G^H y on the K x K grid."""
    return (op.GH @ np.asarray(y)).reshape(op.K, op.K)


def normal(op: nu.Operator, H, x) -> np.ndarray:
    """Re{Z^H F^H H F Z x}."""
    Xh = nu.dft2(nu.zero_pad(op.gs, x)).ravel()
    return nu.zero_pad_adjoint(op.gs, nu.dft2_adjoint((H @ Xh).reshape(op.K, op.K))).real


def gradient(op: nu.Operator, H, b, x) -> np.ndarray:
    """Re{Z^H F^H (H F Z x - b)} with b = G^H y: the gradient of 1/2 ||Phi x - y||^2."""
    Xh = nu.dft2(nu.zero_pad(op.gs, x)).ravel()
    return nu.zero_pad_adjoint(op.gs, nu.dft2_adjoint((H @ Xh).reshape(op.K, op.K) - b)).real
