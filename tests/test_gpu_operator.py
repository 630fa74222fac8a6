"""GPU parity of the measurement operator (Eq. 1) and gradient step (App. A) vs the FP64 oracle.

Tolerance: relative L2 <= 1e-5 for FP32 weights (the operator bound stated
for this path); the oracle is FP64, the GPU path FP32 with FP32 accumulation.
"""
import numpy as np
import pytest

import synth
from oracle import fb as ofb
from oracle import nufft as onu

from gpu_common import pnp, rel_l2, require_gpu, to_dev_c64, to_dev_f32, to_host, torch

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _problem(n, K, M, with_w=False, seed=0, omega_span=0.8):
    rng = np.random.default_rng(100 + seed)
    omega = rng.uniform(-omega_span * np.pi, omega_span * np.pi, (M, 2))
    x = np.maximum(rng.standard_normal((n, n)), 0) + 0.1
    if not with_w:
        return dict(omega=omega, w=None, dl=0.0, Jr=None, x=x, rng=rng)
    w = rng.uniform(-1.0, 1.0, M)
    dl = np.sqrt(4.0 / (n * K))
    Jr = synth.j_per_row_by_w_quartile(w)
    return dict(omega=omega, w=w, dl=dl, Jr=Jr, x=x, rng=rng)


def _plans(pr, n, K, **kw):
    gpu = pnp.Plan(n, K, pr["omega"], pr["w"], pr["dl"], pr["Jr"], **kw)
    ora = onu.Operator(n, K, pr["omega"], pr["w"], pr["dl"], pr["Jr"])
    return gpu, ora


@pytest.mark.parametrize("n,K,M,with_w", [
    (64, 128, 20000, False),     # KB rows, several tiles
    (50, 128, 7001, False),      # ragged image side, odd M
    (64, 128, 20000, True),      # w-folded rows J in {7, 9, 12, 16}
    (96, 256, 30000, True),
    (256, 512, 200000, False),   # the 256^2 / 512^2 / M = 2e5 plain workload
])
def test_phi_forward_parity(n, K, M, with_w):
    pr = _problem(n, K, M, with_w)
    gpu, ora = _plans(pr, n, K)
    y = to_host(gpu.phi_forward(to_dev_f32(pr["x"])))
    assert gpu.device_status() == 0
    assert rel_l2(y, ora.forward(pr["x"])) <= TOL


@pytest.mark.parametrize("n,K,M,with_w", [(64, 128, 20000, False), (50, 128, 7001, True),
                                          (256, 512, 200000, False)])
def test_phi_adjoint_parity(n, K, M, with_w):
    pr = _problem(n, K, M, with_w, seed=1)
    gpu, ora = _plans(pr, n, K)
    r = synth.complex_normal(M, pr["rng"])
    x = to_host(gpu.phi_adjoint(to_dev_c64(r)))
    assert rel_l2(x, ora.adjoint(r)) <= TOL


@pytest.mark.parametrize("n,K,M,with_w", [(64, 128, 20000, False), (64, 128, 20000, True),
                                          (128, 256, 60000, True)])
def test_grad_step_parity(n, K, M, with_w):
    pr = _problem(n, K, M, with_w, seed=2)
    gpu, ora = _plans(pr, n, K)
    y = ora.forward(pr["x"] * 1.3) + 0.1 * synth.complex_normal(M, pr["rng"])
    gamma = 1.0 / M
    out = to_host(gpu.grad_step(to_dev_f32(pr["x"]), to_dev_c64(y), gamma))
    assert gpu.device_status() == 0
    ref = ofb.gradient_step(ora, pr["x"], y, gamma)
    # compare the gradient part, which carries all the operator arithmetic
    assert rel_l2((pr["x"] - out) / gamma, (pr["x"] - ref) / gamma) <= TOL


def test_rows_of_G_match_oracle():
    n, K, M = 64, 128, 5000
    pr = _problem(n, K, M, with_w=True, seed=3)
    gpu, _ = _plans(pr, n, K)
    rows = np.arange(0, M, 7)
    off, wts, cols = gpu.export_rows(rows)
    G = onu.degridding_matrix(onu.GridSpec(n, K), pr["omega"], pr["w"], pr["dl"], pr["Jr"], rows)
    for i in range(rows.size):
        gc = cols[off[i]:off[i + 1]]
        gw = wts[off[i]:off[i + 1]]
        o = np.argsort(gc)
        ref = G[i]
        assert np.array_equal(gc[o], ref.indices[np.argsort(ref.indices)])
        rw = ref.data[np.argsort(ref.indices)]
        assert np.max(np.abs(gw[o] - rw)) <= 1e-6 * np.max(np.abs(rw))


@pytest.mark.parametrize("K", [64, 128, 256, 1024, 2048, 4096, 8192, 16384])
def test_every_fft_size_against_direct_nudft(K):
    # tiny image on every supported grid size: the direct NUDFT is the ground truth
    n, M = 8, 3000
    rng = np.random.default_rng(K)
    omega = rng.uniform(-np.pi, np.pi, (M, 2))   # full range: exercises wrap-around
    x = rng.random((n, n))
    plan = pnp.Plan(n, K, omega)
    y = to_host(plan.phi_forward(to_dev_f32(x)))
    assert rel_l2(y, onu.nudft(omega, x)) <= TOL
    r = synth.complex_normal(M, rng)
    xa = to_host(plan.phi_adjoint(to_dev_c64(r)))
    assert rel_l2(xa, onu.nudft_adjoint(omega, r, n).real) <= TOL


@pytest.mark.parametrize("K", [64, 128, 256, 512, 1024, 2048, 4096, 8192])
def test_twofold_oversampled_sizes_against_oracle(K):
    """n = K/2, the oversampling of every workload: the FFT passes split each length-K transform into
    two length-n ones (no transform over zero padding); forward and adjoint against the FP64 oracle."""
    n, M = K // 2, 3000
    rng = np.random.default_rng(K + 1)
    omega = rng.uniform(-np.pi, np.pi, (M, 2))
    x = rng.random((n, n))
    plan = pnp.Plan(n, K, omega)
    ora = onu.Operator(n, K, omega)
    assert rel_l2(to_host(plan.phi_forward(to_dev_f32(x))), ora.forward(x)) <= TOL
    r = synth.complex_normal(M, rng)
    assert rel_l2(to_host(plan.phi_adjoint(to_dev_c64(r))), ora.adjoint(r)) <= TOL


def test_op_norm_parity():
    n, K, M = 64, 128, 20000
    pr = _problem(n, K, M, seed=4)
    gpu, ora = _plans(pr, n, K)
    v0 = pr["rng"].standard_normal((n, n))
    L_ref, _, _ = ofb.power_iteration(ora, v0, 2000, 1e-12)
    L, it = gpu.op_norm(to_dev_f32(v0), 2000, 1e-8)
    assert abs(L - L_ref) / L_ref <= TOL
    assert L >= 0.999 * M                              # psf peak bound: L >= beta ~ M


def test_empty_operator():
    n, K = 16, 64
    plan = pnp.Plan(n, K, np.zeros((0, 2)))
    x = to_dev_f32(np.ones((n, n)))
    y = plan.phi_forward(x)
    assert y.numel() == 0
    out = to_host(plan.grad_step(x, y, 0.5))
    assert np.array_equal(out, np.ones((n, n)))
    xa = to_host(plan.phi_adjoint(y))
    assert np.array_equal(xa, np.zeros((n, n)))
    choice = plan.autotune(reps=1)       # nothing to time: the defaults stay
    assert choice["gridding_ms"] == -1.0 and choice["run_max"] == plan.info["run_max"]


def test_invalid_arguments_raise():
    with pytest.raises(pnp.PnPError):
        pnp.Plan(15, 64, np.zeros((4, 2)))           # odd n
    with pytest.raises(pnp.PnPError):
        pnp.Plan(16, 100, np.zeros((4, 2)))          # K not a power of two
    with pytest.raises(pnp.PnPError):
        pnp.Plan(16, 64, np.zeros((4, 2)), J_per_row=np.full(4, 20, np.int8))
    with pytest.raises(pnp.PnPError):
        pnp.Plan(16, 64, np.full((4, 2), np.nan))


def test_adjoint_identity_on_gpu():
    n, K, M = 128, 256, 50000
    pr = _problem(n, K, M, with_w=True, seed=5)
    gpu, _ = _plans(pr, n, K)
    x = pr["rng"].standard_normal((n, n))
    r = synth.complex_normal(M, pr["rng"])
    yx = to_host(gpu.phi_forward(to_dev_f32(x)))
    xr = to_host(gpu.phi_adjoint(to_dev_c64(r)))
    lhs = np.vdot(r, yx).real
    rhs = np.sum(x * xr)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(yx) * np.linalg.norm(r)


def test_fused_grad_equals_forward_then_adjoint():
    n, K, M = 128, 256, 50000
    pr = _problem(n, K, M, with_w=True, seed=6)
    gpu, _ = _plans(pr, n, K)
    x = to_dev_f32(pr["x"])
    y = to_dev_c64(synth.complex_normal(M, pr["rng"]))
    g1 = to_host(gpu.grad_step(x, y, 1.0))
    r = gpu.phi_forward(x) - y
    g2 = pr["x"] - to_host(gpu.phi_adjoint(r.contiguous()))
    assert rel_l2(pr["x"] - g1, pr["x"] - g2) <= 1e-5


def test_unit_size_does_not_change_result():
    n, K, M = 64, 128, 20000
    pr = _problem(n, K, M, with_w=True, seed=7)
    gpu, _ = _plans(pr, n, K)
    x = to_dev_f32(pr["x"])
    y0 = to_host(gpu.phi_forward(x))
    gpu.set_unit_nnz(700)
    y1 = to_host(gpu.phi_forward(x))
    assert rel_l2(y1, y0) <= 1e-6


@pytest.mark.parametrize("row_batch", [1, 2, 4])
def test_row_batch_matches_oracle(row_batch):
    """Residuals formed 1, 2 or 4 rows at a time: same pairing of the warp sums, so the
    de-gridded rows agree bit for bit and the fused gradient matches the oracle."""
    n, K, M = 128, 256, 60000
    pr = _problem(n, K, M, with_w=True, seed=11)
    # rows clustered on 2000 cells with the same fractional offset, so that long runs of
    # rows sharing a tap window (cut at the run cap) and partial last batches both occur
    rng = pr["rng"]
    cells = rng.integers(-K // 3, K // 3, (2000, 2))
    kap = cells[rng.integers(0, 2000, M)] + rng.uniform(0.6, 0.7, (M, 2))
    pr["omega"] = 2 * np.pi * kap / K
    gpu, ora = _plans(pr, n, K)
    yh = ora.forward(pr["x"] * 0.7) + 0.05 * synth.complex_normal(M, pr["rng"])
    x, y = to_dev_f32(pr["x"]), to_dev_c64(yh)
    gpu.set_row_batch(1)
    y1 = to_host(gpu.phi_forward(x))
    gpu.set_row_batch(row_batch)
    assert gpu.info["row_batch"] == row_batch
    yb = to_host(gpu.phi_forward(x))
    assert np.array_equal(yb, y1)
    assert rel_l2(yb, ora.forward(pr["x"])) <= TOL
    gamma = 1.0 / M
    g = to_host(gpu.grad_step(x, y, gamma))
    assert gpu.device_status() == 0
    ref = ofb.gradient_step(ora, pr["x"], yh, gamma)
    assert rel_l2((pr["x"] - g) / gamma, (pr["x"] - ref) / gamma) <= TOL


def test_autotune_keeps_results_and_reports_its_choice():
    """The tuner only changes the work list: gradient steps agree up to summation order."""
    n, K, M = 64, 128, 20000
    pr = _problem(n, K, M, with_w=True, seed=9)
    gpu, ora = _plans(pr, n, K)
    yh = ora.forward(pr["x"] * 1.3) + 0.1 * synth.complex_normal(M, pr["rng"])
    x, y = to_dev_f32(pr["x"]), to_dev_c64(yh)
    gamma = 1.0 / M
    g0 = to_host(gpu.grad_step(x, y, gamma))
    choice = gpu.autotune(reps=1)
    assert choice["run_max"] in (3, 4, 6, 8) and choice["unit_nnz"] in (1 << 16, 1 << 17, 1 << 18)
    assert choice["gridding_ms"] > 0
    info = gpu.info
    assert (info["run_max"], info["unit_nnz"]) == (choice["run_max"], choice["unit_nnz"])
    assert choice["row_batch"] in (1, 2, 4) and info["row_batch"] == choice["row_batch"]
    g1 = to_host(gpu.grad_step(x, y, gamma))
    assert gpu.device_status() == 0
    assert rel_l2((pr["x"] - g1) / gamma, (pr["x"] - g0) / gamma) <= 1e-6
    ref = ofb.gradient_step(ora, pr["x"], yh, gamma)
    assert rel_l2((pr["x"] - g1) / gamma, (pr["x"] - ref) / gamma) <= TOL


def test_bf16_weights_error_is_bounded():
    n, K, M = 64, 128, 20000
    pr = _problem(n, K, M, with_w=True, seed=8)
    gpu = pnp.Plan(n, K, pr["omega"], pr["w"], pr["dl"], pr["Jr"], weight_dtype="bf16")
    ora = onu.Operator(n, K, pr["omega"], pr["w"], pr["dl"], pr["Jr"])
    y = to_host(gpu.phi_forward(to_dev_f32(pr["x"])))
    err = rel_l2(y, ora.forward(pr["x"]))
    assert err <= 2.0 ** -8          # one BF16 rounding per weight, averaged over the row


@pytest.mark.parametrize("case", ["narrow_band", "single_edge_row", "two_rows"])
def test_fft_pruned_to_the_uv_support(case):
    """The split FFT passes transform and move only G's uv support (the band of grid rows k1 that hold
    taps and, per row, the cells up to the largest centred |k0| of a tap): an asymmetric narrow band,
    one row whose taps wrap around both grid edges, and two rows far apart.  Forward, adjoint and the
    fused gradient against the oracle, each twice with different inputs, so that a cell left stale
    outside the support by one call would show in the next."""
    n, K = 128, 256
    rng = np.random.default_rng(41)
    if case == "narrow_band":
        M = 4000
        omega = np.stack([rng.uniform(-np.pi, np.pi, M), rng.uniform(-0.15 * np.pi, 0.1 * np.pi, M)], axis=1)
    elif case == "single_edge_row":
        M = 1
        omega = np.array([[0.995 * np.pi, -0.995 * np.pi]])
    else:
        M = 2
        omega = np.array([[0.1, 0.7 * np.pi], [-0.6 * np.pi, -0.2]])
    gpu = pnp.Plan(n, K, omega)
    ora = onu.Operator(n, K, omega)
    for rep in range(2):
        x = rng.random((n, n)) + rep
        assert rel_l2(to_host(gpu.phi_forward(to_dev_f32(x))), ora.forward(x)) <= TOL
        r = synth.complex_normal(M, rng)
        assert rel_l2(to_host(gpu.phi_adjoint(to_dev_c64(r))), ora.adjoint(r)) <= TOL
        y = -ora.forward(x) + synth.complex_normal(M, rng)   # a residual without cancellation (M may be 1)
        out = to_host(gpu.grad_step(to_dev_f32(x), to_dev_c64(y), 0.5))
        ref = ofb.gradient_step(ora, x, y, 0.5)
        assert rel_l2(x - out, x - ref) <= TOL
    assert gpu.device_status() == 0
