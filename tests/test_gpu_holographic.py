"""GPU holographic normal operator H = G^H G (App. E, Eq. phidagphi) against the oracle."""
import numpy as np
import pytest

import synth
from oracle import fb as ofb
from oracle import holographic as oh
from oracle import nufft as onu

from gpu_common import PnPError_type, pnp, rel_l2, require_gpu, to_dev_c64, to_dev_f32, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _problem(n, K, M, with_w, seed):
    rng = np.random.default_rng(600 + seed)
    omega = rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (M, 2))
    x = np.maximum(rng.standard_normal((n, n)), 0) + 0.1
    if not with_w:
        return dict(omega=omega, w=None, dl=0.0, Jr=None, x=x, rng=rng)
    w = rng.uniform(-1.0, 1.0, M)
    return dict(omega=omega, w=w, dl=np.sqrt(4.0 / (n * K)), Jr=synth.j_per_row_by_w_quartile(w), x=x, rng=rng)


@pytest.mark.parametrize("n,K,M,with_w", [
    (64, 128, 20000, False),
    (48, 128, 15000, True),       # w-folded rows J in {7, 9, 12, 16}: stencils of 31 x 31
    (32, 64, 200000, False),      # many rows per cell: H is far smaller than G
])
def test_holographic_fb_matches_oracle(n, K, M, with_w):
    pr = _problem(n, K, M, with_w, n + M)
    ora = onu.Operator(n, K, pr["omega"], pr["w"], pr["dl"], pr["Jr"])
    y = ora.forward(pr["x"]) + 0.05 * synth.complex_normal(M, pr["rng"])
    L, _, _ = ofb.power_iteration(ora, pr["rng"].standard_normal((n, n)), 1000, 1e-10)
    gamma, t, iters = ofb.step_size(L), 1e-3, 30
    x_ref, _ = ofb.pnp_fb(ora, y, gamma, lambda z: ofb.haar_denoise(z, t), iters)
    plan = pnp.Plan(n, K, pr["omega"], pr["w"], pr["dl"], pr["Jr"])
    plan.set_holographic(True)
    S = 2 * (16 if with_w else 7) - 1
    assert plan.info["holographic_bytes"] == S * S * K * K * 8
    x, st = plan.fb_run(pnp.HaarDenoiser(t), to_dev_c64(y), gamma=gamma, L=L, max_iter=iters, check_every=10)
    assert st.iters == iters and plan.device_status() == 0
    assert rel_l2(to_host(x), x_ref) <= 1e-4
    # the holographic normal operator drives the power iteration as the plain one does
    v0 = pr["rng"].standard_normal((n, n))
    Lh, _ = plan.op_norm(to_dev_f32(v0), 100, 0.0)
    plan.set_holographic(False)
    Lg, _ = plan.op_norm(to_dev_f32(v0), 100, 0.0)
    L_ref, _, _ = ofb.power_iteration(ora, v0, 100, 0.0)
    assert abs(Lh - L_ref) <= 1e-5 * L_ref and abs(Lg - L_ref) <= 1e-5 * L_ref


def test_holographic_normal_operator_against_the_oracle_matrix():
    n, K, M = 32, 64, 5000
    pr = _problem(n, K, M, True, 7)
    ora = onu.Operator(n, K, pr["omega"], pr["w"], pr["dl"], pr["Jr"])
    H = oh.holographic_matrix(ora)
    plan = pnp.Plan(n, K, pr["omega"], pr["w"], pr["dl"], pr["Jr"])
    plan.set_holographic(True)
    v0 = pr["rng"].standard_normal((n, n))
    L, _ = plan.op_norm(to_dev_f32(v0), 1, 0.0)          # one application: ||Re{Z^H F^H H F Z v}||
    v = v0 / np.linalg.norm(v0)
    assert L == pytest.approx(np.linalg.norm(oh.normal(ora, H, v)), rel=1e-5)


def test_stacked_plans_have_no_holographic_form():
    n, K, M = 32, 64, 3000
    pr = _problem(n, K, M, True, 9)
    stk, cen = synth.w_stacks(pr["w"], 2)
    plan = pnp.Plan(n, K, pr["omega"], pr["w"], pr["dl"], synth.j_per_row_stacked(pr["w"], stk, cen, pr["w"]),
                    stack=stk, w_centres=cen)
    with pytest.raises(PnPError_type()):
        plan.set_holographic(True)
