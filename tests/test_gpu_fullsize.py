"""Full-size parity of the operator at the benchmark workloads, on sampled outputs.

Workloads: 2048^2 image / 4096^2 grid and 4096^2 image / 8192^2 grid, M = 2e7
MeerKAT-like rows with w folded into G, J in {7, 9, 12, 16} by |w| quartile
(64 radial data blocks for the 4096^2 case), complex64 weights.  The oracle
evaluates y = G F Z x only on seeded sampled rows (its FFT runs at full size);
the adjoint is checked through the identity <Phi x, r> = <x, Phi^H r> and the
fused gradient through forward-then-adjoint, both at full size.
"""
import numpy as np
import pytest

import synth
from oracle import nufft as onu
from oracle import wstack as ows

from gpu_common import pnp, rel_l2, require_gpu, to_dev_c64, to_dev_f32, to_host, torch

pytestmark = pytest.mark.gpu

CASES = {"2048": ("C1", 2048, 4096, 1), "4096": ("C3", 4096, 8192, 64)}


@pytest.fixture(scope="module", params=sorted(CASES))
def full(request):
    require_gpu()
    name, n, K, nb = CASES[request.param]
    prob = synth.make_problem(name)
    plan = pnp.Plan(n, K, prob["omega"], prob["w"], prob["dl"], prob["J_per_row"],
                    block=prob["block"], nblocks=nb)
    yield prob, plan
    plan.close()
    torch.cuda.empty_cache()


def test_sampled_rows_forward(full):
    prob, plan = full
    n, K, M = prob["n"], prob["K"], prob["M"]
    x = prob["x_true"]
    y = plan.phi_forward(to_dev_f32(x))
    rows = np.sort(synth.rng_for("misc").choice(M, 2000, replace=False))
    y_s = to_host(y[torch.from_numpy(rows).cuda()])
    gs = onu.GridSpec(n, K)
    Xhat = onu.dft2(onu.zero_pad(gs, x)).ravel()
    G = onu.degridding_matrix(gs, prob["omega"], prob["w"], prob["dl"], prob["J_per_row"], rows)
    assert rel_l2(y_s, G @ Xhat) <= 1e-5


def test_sampled_rows_adjoint_elementwise(full):
    """Phi^H r at full size, element by element, for r zero except on 2000 seeded rows that include
    the 500 rows in the densest uv cells: the whole work list runs (every tile, block and support)
    and the oracle forms Re{Z^H F^H G_rows^H r_rows} with its full-size FFT."""
    prob, plan = full
    n, K, M = prob["n"], prob["K"], prob["M"]
    om = prob["omega"]
    k = np.floor(om * (K / (2 * np.pi))).astype(np.int64) % K
    cell = k[:, 0] * K + k[:, 1]
    occupancy = np.bincount(cell, minlength=K * K)[cell]
    dense = np.argsort(-occupancy, kind="stable")[:500]
    rest = np.setdiff1d(np.arange(M), dense)
    rows = np.sort(np.concatenate([dense, synth.rng_for("misc").choice(rest, 1500, replace=False)]))
    r = np.zeros(M, dtype=np.complex128)
    r[rows] = synth.complex_normal(rows.size, np.random.default_rng(31))
    xg = to_host(plan.phi_adjoint(to_dev_c64(r)))
    gs = onu.GridSpec(n, K)
    G = onu.degridding_matrix(gs, om, prob["w"], prob["dl"], prob["J_per_row"], rows)
    grid = (G.conj().T @ r[rows]).reshape(K, K)
    ref = onu.zero_pad_adjoint(gs, onu.dft2_adjoint(grid)).real
    assert rel_l2(xg, ref) <= 1e-5


def test_adjoint_identity_full(full):
    prob, plan = full
    rng = np.random.default_rng(9)
    x = rng.standard_normal((prob["n"], prob["n"])).astype(np.float32)
    r = prob["noise"]
    yx = to_host(plan.phi_forward(to_dev_f32(x)))
    xr = to_host(plan.phi_adjoint(to_dev_c64(r)))
    lhs = np.vdot(r, yx).real
    rhs = float(np.sum(x.astype(np.float64) * xr))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(yx) * np.linalg.norm(r)


def test_fused_gradient_full(full):
    prob, plan = full
    x = to_dev_f32(prob["x_true"])
    y = to_dev_c64(prob["noise"])
    g1 = plan.grad_step(x, y, 1.0)
    r = plan.phi_forward(x) - y
    g2 = x - plan.phi_adjoint(r.contiguous())
    assert rel_l2(to_host(x - g1), to_host(x - g2)) <= 1e-5


@pytest.fixture(scope="module")
def stacked():
    """The 4096^2 / 8192^2 / M = 2e7 workload as an 8-stack w-stacked operator (minimum-taps layout)."""
    require_gpu()
    prob = synth.make_problem("C3", n_stacks=8)
    plan = pnp.Plan(prob["n"], prob["K"], prob["omega"], prob["w"], prob["dl"], prob["J_per_row"],
                    block=prob["block"], nblocks=64, stack=prob["stack"], w_centres=prob["w_centres"])
    yield prob, plan
    plan.close()
    torch.cuda.empty_cache()


def test_stacked_sampled_rows_forward(stacked):
    prob, plan = stacked
    x = prob["x_true"]
    y = plan.phi_forward(to_dev_f32(x))
    # rows of two stacks (an outer and an inner one): two full-size FFTs on the oracle side
    st = prob["stack"]
    pick = np.nonzero((st == 0) | (st == 4))[0]
    rows = np.sort(synth.rng_for("misc").choice(pick, 2000, replace=False))
    y_s = to_host(y[torch.from_numpy(rows).cuda()])
    ref = ows.forward_rows(prob["n"], prob["K"], prob["omega"], prob["w"], prob["dl"], st, prob["w_centres"],
                           prob["J_per_row"], x, rows)
    assert rel_l2(y_s, ref) <= 1e-5


def test_stacked_adjoint_and_gradient_full(stacked):
    prob, plan = stacked
    rng = np.random.default_rng(19)
    x = rng.standard_normal((prob["n"], prob["n"])).astype(np.float32)
    r = prob["noise"]
    yx = to_host(plan.phi_forward(to_dev_f32(x)))
    xr = to_host(plan.phi_adjoint(to_dev_c64(r)))
    lhs = np.vdot(r, yx).real
    rhs = float(np.sum(x.astype(np.float64) * xr))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(yx) * np.linalg.norm(r)
    xd, yd = to_dev_f32(prob["x_true"]), to_dev_c64(prob["noise"])
    g1 = plan.grad_step(xd, yd, 1.0)
    g2 = xd - plan.phi_adjoint((plan.phi_forward(xd) - yd).contiguous())
    assert rel_l2(to_host(xd - g1), to_host(xd - g2)) <= 1e-5
