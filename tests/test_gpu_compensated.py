"""Compensated summation in the gridding pass (G^H r of App. A, summed over many rows per cell as
in Eq. phidagphi).  In a dense uv core thousands of rows meet in one grid cell; the 128^2 image /
256^2 grid / M = 2e6 layout of the 256^2 configuration's kind (8 h track, KB J = 7) puts up to
~11,000 rows (~5e5 taps) in a cell.  The adjoint of seeded random residuals is compared with the
FP64 oracle element by element with the compensated flush on and off: on, it meets the operator
tolerance, and its error is a fraction of the plain FP32 sums' error.
"""
import numpy as np
import pytest

import synth
from oracle import nufft as onu

from gpu_common import pnp, rel_l2, require_gpu, to_dev_c64, to_host, torch

pytestmark = pytest.mark.gpu


def test_compensated_gridding_reduces_dense_core_error():
    require_gpu()
    n, K, M = 128, 256, 2_000_000
    prob = synth.make_problem("C0", M=M, n=n, K=K)
    r = synth.complex_normal(M, np.random.default_rng(77))
    ref = onu.Operator(n, K, prob["omega"]).adjoint(r)
    plan = pnp.Plan(n, K, prob["omega"])
    rd = to_dev_c64(r)
    assert plan.info["compensated"] == 1
    errs = {}
    for on in (True, False):
        plan.set_compensated(on)
        errs[on] = max(rel_l2(to_host(plan.phi_adjoint(rd)), ref) for _ in range(3))
    print(f"dense-core adjoint rel L2: compensated {errs[True]:.3e}, plain FP32 {errs[False]:.3e}")
    assert errs[True] <= 1e-5
    assert errs[True] <= 0.5 * errs[False]
    plan.close()
    torch.cuda.empty_cache()
