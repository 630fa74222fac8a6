"""Compensated summation in the gridding pass (G^H r of App. A, summed over many rows per cell as
in Eq. phidagphi).  In a dense uv core thousands of rows meet in one grid cell: the 128^2 image /
256^2 grid / M = 2e6 layout of the 256^2 configuration's kind (8 h track, KB J = 7) in 64 radial
data blocks puts up to ~11,000 rows (~5e5 taps) in a cell.  The adjoint is compared with the FP64
oracle element by element with the compensated flush on and off, for two residuals:

* seeded random residuals: the FP32 partial sums carry random-sign errors that stay at the level of
  the FP32 FFT (~3e-7), so both pass the operator tolerance and the compensated one is no worse;
* residuals of opposite sign in alternate data blocks (each work unit holds one block): the work
  units' partial sums at the dense core are large and cancel in the grid, the case compensation is
  for; there the plain FP32 sums lose accuracy and the compensated ones do not.
"""
import numpy as np
import pytest

import synth
from oracle import nufft as onu

from gpu_common import pnp, rel_l2, require_gpu, to_dev_c64, to_host, torch

pytestmark = pytest.mark.gpu


def test_compensated_gridding_in_a_dense_core():
    require_gpu()
    n, K, M = 128, 256, 2_000_000
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    block = synth.radial_blocks(prob["omega"], 64, synth.rng_for("blocks"))
    ora = onu.Operator(n, K, prob["omega"])
    plan = pnp.Plan(n, K, prob["omega"], block=block, nblocks=64)
    assert plan.info["compensated"] == 1
    rng = np.random.default_rng(77)
    cases = {"random": synth.complex_normal(M, rng),
             "cancelling": np.where(block % 2 == 0, 1.0, -1.0) * (1.0 + 0.01 * synth.complex_normal(M, rng))}
    errs = {}
    for name, r in cases.items():
        ref = ora.adjoint(r)
        rd = to_dev_c64(r)
        for on in (True, False):
            plan.set_compensated(on)
            errs[name, on] = max(rel_l2(to_host(plan.phi_adjoint(rd)), ref) for _ in range(3))
        print(f"dense-core adjoint rel L2, {name} residuals: compensated {errs[name, True]:.3e}, "
              f"plain FP32 {errs[name, False]:.3e}")
    assert errs["random", True] <= 1e-5 and errs["random", False] <= 1e-5
    assert errs["random", True] <= 1.2 * errs["random", False]
    assert errs["cancelling", True] <= 1e-5
    assert errs["cancelling", True] <= 0.5 * errs["cancelling", False]
    plan.close()
    torch.cuda.empty_cache()
