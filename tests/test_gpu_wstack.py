"""GPU parity of the w-stacked operator (App. E, Eq. phip / phidagphi) against the stacked oracle."""
import numpy as np
import pytest

import synth
from oracle import fb as ofb
from oracle import nufft as onu
from oracle.wstack import StackedOperator

from gpu_common import pnp, rel_l2, require_gpu, to_dev_c64, to_dev_f32, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _problem(n, K, M, P, seed=0, empty=None):
    rng = np.random.default_rng(500 + seed)
    omega = rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (M, 2))
    w = rng.uniform(-1.0, 1.0, M)
    dl = np.sqrt(8.0 / (n * K))              # largest |w| spreads 8 cells
    stack, cen = synth.w_stacks(w, P)
    if empty is not None:                    # a stack with no rows: its rows go to the next one
        stack[stack == empty] = (empty + 1) % P
    Jr = synth.j_per_row_stacked(w, stack, cen, w)
    x = np.maximum(rng.standard_normal((n, n)), 0) + 0.1
    gpu = pnp.Plan(n, K, omega, w, dl, Jr, stack=stack, w_centres=cen)
    ora = StackedOperator(n, K, omega, w, dl, stack, cen, Jr)
    return dict(omega=omega, w=w, dl=dl, stack=stack, cen=cen, Jr=Jr, x=x, rng=rng, gpu=gpu, ora=ora)


@pytest.mark.parametrize("n,K,M,P,empty", [
    (64, 128, 20000, 2, None),
    (96, 256, 40000, 4, None),       # several tiles, ragged image side for the tile grid
    (64, 128, 20000, 3, 1),          # a stack with no rows
])
def test_stacked_forward_adjoint_gradient(n, K, M, P, empty):
    pr = _problem(n, K, M, P, seed=P, empty=empty)
    gpu, ora = pr["gpu"], pr["ora"]
    assert gpu.info["nstacks"] == P
    x = pr["x"]
    y = to_host(gpu.phi_forward(to_dev_f32(x)))
    assert rel_l2(y, ora.forward(x)) <= TOL
    r = synth.complex_normal(M, pr["rng"])
    xa = to_host(gpu.phi_adjoint(to_dev_c64(r)))
    assert rel_l2(xa, ora.adjoint(r)) <= TOL
    yh = ora.forward(x * 1.2) + 0.05 * synth.complex_normal(M, pr["rng"])
    gamma = 1.0 / M
    g = to_host(gpu.grad_step(to_dev_f32(x), to_dev_c64(yh), gamma))
    ref = ofb.gradient_step(ora, x, yh, gamma)
    assert rel_l2((x - g) / gamma, (x - ref) / gamma) <= TOL
    assert gpu.device_status() == 0


def test_one_stack_at_zero_is_the_plain_plan():
    n, K, M = 64, 128, 20000
    rng = np.random.default_rng(77)
    omega = rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (M, 2))
    w = rng.uniform(-1.0, 1.0, M)
    dl = np.sqrt(4.0 / (n * K))
    Jr = synth.j_per_row_by_w_quartile(w)
    x = to_dev_f32(rng.random((n, n)))
    a = pnp.Plan(n, K, omega, w, dl, Jr)
    b = pnp.Plan(n, K, omega, w, dl, Jr, stack=np.zeros(M, dtype=np.int32), w_centres=[0.0])
    assert np.array_equal(to_host(a.phi_forward(x)), to_host(b.phi_forward(x)))


def test_stacked_op_norm_and_fb_parity():
    n, K, M, P = 64, 128, 20000, 4
    pr = _problem(n, K, M, P, seed=9)
    gpu, ora = pr["gpu"], pr["ora"]
    v0 = pr["rng"].standard_normal((n, n))
    # the same number of power iterations on both sides: the estimates then agree to the FP32
    # rounding of the operator, whatever the gap between the top eigenvalues
    L_ref, _, _ = ofb.power_iteration(ora, v0, 200, 0.0)
    L, it = gpu.op_norm(to_dev_f32(v0), 200, 0.0)
    assert it == 200
    assert abs(L - L_ref) / L_ref <= TOL
    x_true = pr["x"]
    y = ora.forward(x_true) + 1e-3 * synth.complex_normal(M, pr["rng"])
    gamma = ofb.step_size(L_ref)
    t = 1e-3
    iters = 50
    x_ref, _ = ofb.pnp_fb(ora, y, gamma, lambda z: ofb.haar_denoise(z, t), iters)
    x, st = gpu.fb_run(pnp.HaarDenoiser(t), to_dev_c64(y), gamma=gamma, L=L, max_iter=iters, check_every=10)
    assert st.iters == iters
    assert rel_l2(to_host(x), x_ref) <= 1e-4


def test_stacking_matches_plain_rows_of_full_support():
    """Stacked rows of small support approximate the same operator as unstacked rows of large
    support (both against the paraxial direct NUDFT on a small case)."""
    n, K, M, P = 32, 64, 3000, 4
    pr = _problem(n, K, M, P, seed=12)
    x = pr["x"]
    yd = onu.nudft(pr["omega"], x, pr["w"], pr["dl"], paraxial=True)
    ys = to_host(pr["gpu"].phi_forward(to_dev_f32(x)))
    plain = pnp.Plan(n, K, pr["omega"], pr["w"], pr["dl"], synth.j_per_row_by_w_quartile(pr["w"]))
    yp = to_host(plain.phi_forward(to_dev_f32(x)))
    es, ep = rel_l2(ys, yd), rel_l2(yp, yd)
    assert es < 2e-2 and ep < 2e-2
    assert pr["gpu"].info["nnz"] < 0.5 * plain.info["nnz"]
