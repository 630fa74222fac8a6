"""Compensated summation in the gridding pass (G^H r of App. A, summed over many rows per cell as
in Eq. phidagphi).  The adjoint is compared with the FP64 oracle element by element with the
compensated flush on and off, in dense uv cores of the 256^2 configuration's kind (8 h track,
KB J = 7):

* seeded random residuals, 128^2 image / 256^2 grid / M = 2e6 (up to ~11,000 rows in a cell): the
  random-sign rounding errors of the FP32 sums stay at the level of the FP32 FFT, both pass the
  operator tolerance and the compensated sums are no worse;
* the dirty beam (r = 1, the quantity App. F's normalisation beta and the dirty-peak bound alpha
  are read from), 256^2 image / 512^2 grid / M = 2e7 (76 rows per cell on average): every term at
  the dense core has the same sign, the core dominates the image, and each core cell receives the
  partial sums of many work units; there the plain FP32 flush loses accuracy and the compensated
  one does not.
"""
import numpy as np
import pytest

import synth
from oracle import nufft as onu

from gpu_common import pnp, rel_l2, require_gpu, to_dev_c64, to_host, torch

pytestmark = pytest.mark.gpu


def _oracle_adjoint_chunked(n, K, omega, r, chunk=2_000_000):
    """Re{Z^H F^H G^H r} with G built and applied chunk by chunk of rows (FP64)."""
    gs = onu.GridSpec(n, K)
    grid = np.zeros(K * K, dtype=np.complex128)
    for s in range(0, omega.shape[0], chunk):
        rows = np.arange(s, min(s + chunk, omega.shape[0]))
        G = onu.degridding_matrix(gs, omega, rows=rows)
        grid += G.conj().T @ r[rows]
    return onu.zero_pad_adjoint(gs, onu.dft2_adjoint(grid.reshape(K, K))).real


def _errors(plan, r, ref):
    rd = to_dev_c64(r)
    out = {}
    for on in (True, False):
        plan.set_compensated(on)
        out[on] = max(rel_l2(to_host(plan.phi_adjoint(rd)), ref) for _ in range(3))
    return out


def test_compensated_gridding_random_residuals():
    require_gpu()
    n, K, M = 128, 256, 2_000_000
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    plan = pnp.Plan(n, K, prob["omega"])
    assert plan.info["compensated"] == 0   # plain FP32 flush by default
    r = synth.complex_normal(M, np.random.default_rng(77))
    e = _errors(plan, r, _oracle_adjoint_chunked(n, K, prob["omega"], r))
    print(f"dense-core adjoint rel L2, random residuals: compensated {e[True]:.3e}, plain FP32 {e[False]:.3e}")
    assert e[True] <= 1e-5 and e[False] <= 1e-5
    assert e[True] <= 1.2 * e[False]
    plan.close()
    torch.cuda.empty_cache()


def test_compensated_gridding_dirty_beam():
    require_gpu()
    n, K, M = 256, 512, 20_000_000
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    plan = pnp.Plan(n, K, prob["omega"])
    r = np.ones(M, dtype=np.complex128)
    e = _errors(plan, r, _oracle_adjoint_chunked(n, K, prob["omega"], r))
    print(f"dense-core adjoint rel L2, dirty beam: compensated {e[True]:.3e}, plain FP32 {e[False]:.3e}")
    assert e[True] <= 1e-5
    assert e[True] <= 0.5 * e[False]
    plan.close()
    torch.cuda.empty_cache()
