"""Pins of the w-stacked operator oracle (App. E, Eq. phip / phidagphi) and of the stack layout."""
import numpy as np
import pytest

import synth
from oracle import nufft as nu
from oracle.wstack import StackedOperator


def _rng(s=0):
    return np.random.default_rng(3000 + s)


def _problem(n=16, K=32, M=200, seed=0):
    rng = _rng(seed)
    omega = rng.uniform(-0.8 * np.pi, 0.8 * np.pi, (M, 2))
    w = rng.uniform(-1.0, 1.0, M)
    dl = np.sqrt(4.0 / (n * K))            # largest |w| spreads 4 cells
    return omega, w, dl


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_w_stacks_layout():
    w = _rng(1).uniform(-3.0, 5.0, 1001)
    stack, cen = synth.w_stacks(w, 4)
    cnt = np.bincount(stack, minlength=4)
    assert cnt.sum() == w.size and cnt.max() - cnt.min() <= 1
    for s in range(4):
        ws = w[stack == s]
        assert cen[s] == pytest.approx(0.5 * (ws.min() + ws.max()))
        if s:
            assert ws.min() >= w[stack == s - 1].max()        # bins are ordered in w
    one, c1 = synth.w_stacks(w, 1)
    assert not one.any() and c1[0] == pytest.approx(0.5 * (w.min() + w.max()))


def test_stacked_supports_reduce_to_quartile_rule():
    w = _rng(2).uniform(-1.0, 1.0, 999)
    J0 = synth.j_per_row_stacked(w, np.zeros(w.size, dtype=np.int32), np.zeros(1), w)
    assert np.array_equal(J0, synth.j_per_row_by_w_quartile(w))
    stack, cen = synth.w_stacks(w, 4)
    J4 = synth.j_per_row_stacked(w, stack, cen, w)
    # residual |w| <= an eighth of the range (a quarter of the largest |w|): no row needs more than
    # the second support, and G holds well under half the taps of the unstacked rows
    Jq = synth.j_per_row_by_w_quartile(w).astype(np.int64)
    assert J4.max() <= 9
    assert (J4.astype(np.int64) ** 2).sum() < 0.5 * (Jq ** 2).sum()


def test_single_zero_centred_stack_is_the_plain_operator():
    n, K, M = 16, 32, 120
    omega, w, dl = _problem(n, K, M)
    Jr = synth.j_per_row_by_w_quartile(w)
    x = _rng(3).random((n, n))
    ys = StackedOperator(n, K, omega, w, dl, np.zeros(M, dtype=np.int32), [0.0], Jr).forward(x)
    # the unit chirp makes the image complex before the grid correction: equal up to rounding
    assert _rel(ys, nu.Operator(n, K, omega, w, dl, Jr).forward(x)) < 1e-14


def test_untruncated_stacked_rows_equal_untruncated_plain_rows():
    # exp(i pi a_m p^2) = exp(i pi a_p p^2) exp(i pi (a_m - a_p) p^2) on every image pixel, so with
    # whole rows (J_m = K) stacking changes nothing but rounding; a sign or scale slip in the
    # centre chirp or in the residual w breaks this by O(1)
    n, K, M = 16, 32, 150
    omega, w, dl = _problem(n, K, M, seed=4)
    stack, cen = synth.w_stacks(w, 3)
    full = np.full(M, K, dtype=np.int64)
    x = _rng(5).random((n, n))
    op_s = StackedOperator(n, K, omega, w, dl, stack, cen, full)
    ys = op_s.forward(x)
    yp = nu.Operator(n, K, omega, w, dl, full).forward(x)
    assert _rel(ys, yp) < 1e-12
    # and both equal the paraxial direct NUDFT up to the KB interpolation error
    assert _rel(ys, nu.nudft(omega, x, w, dl, paraxial=True)) < 5e-6
    r = _rng(6).standard_normal(M) + 1j * _rng(7).standard_normal(M)
    assert _rel(op_s.adjoint_complex(r), nu.Operator(n, K, omega, w, dl, full).adjoint_complex(r)) < 1e-12


def test_stacked_adjoint_identity():
    n, K, M = 16, 32, 200
    omega, w, dl = _problem(n, K, M, seed=8)
    stack, cen = synth.w_stacks(w, 4)
    Jr = synth.j_per_row_stacked(w, stack, cen, w)
    op = StackedOperator(n, K, omega, w, dl, stack, cen, Jr)
    rng = _rng(9)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    r = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    lhs = np.vdot(r, op.forward(x))
    rhs = np.vdot(op.adjoint_complex(r), x)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(op.forward(x)) * np.linalg.norm(r)
    xr = x.real
    assert np.vdot(r, op.forward(xr)).real == pytest.approx(np.sum(xr * op.adjoint(r)), rel=1e-12)


def test_stacking_lowers_truncation_error_at_fixed_support():
    # the residual chirp left to the rows shrinks with the number of stacks, so at a fixed
    # small support the error against the paraxial NUDFT falls with P
    n, K, M = 16, 32, 300
    omega, w, dl = _problem(n, K, M, seed=10)
    x = _rng(11).random((n, n))
    yd = nu.nudft(omega, x, w, dl, paraxial=True)
    J7 = np.full(M, 7, dtype=np.int64)
    errs = []
    for P in (1, 2, 4, 8):
        stack, cen = synth.w_stacks(w, P)
        errs.append(_rel(StackedOperator(n, K, omega, w, dl, stack, cen, J7).forward(x), yd))
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < errs[0] / 4


def test_min_taps_partition():
    # heavy-tailed w (most rows near 0, long tails): the minimum-taps partition never holds more
    # taps than one stack at 0 and beats equal-count bins
    rng = _rng(12)
    w = rng.standard_t(2, 20000) * 300.0
    qs = synth.j_per_row_by_w_quartile(w).astype(np.int64)
    for P in (2, 3, 4, 8):
        stack, cen = synth.w_stacks_min_taps(w, P)
        assert stack.min() >= 0 and stack.max() < P and cen.size == P
        assert np.all(np.diff(cen) >= 0)
        for s in range(P):                                   # contiguous in w
            if s and (stack == s).any() and (stack == s - 1).any():
                assert w[stack == s].min() >= w[stack == s - 1].max()
        J = synth.j_per_row_stacked(w, stack, cen, w).astype(np.int64)
        assert (J ** 2).sum() <= (qs ** 2).sum()
        se, ce = synth.w_stacks(w, P)
        Je = synth.j_per_row_stacked(w, se, ce, w).astype(np.int64)
        assert (J ** 2).sum() <= (Je ** 2).sum()


def test_forward_rows_equals_the_operator_rows():
    n, K, M = 16, 32, 200
    omega, w, dl = _problem(n, K, M, seed=13)
    stack, cen = synth.w_stacks(w, 3)
    Jr = synth.j_per_row_stacked(w, stack, cen, w)
    x = _rng(14).random((n, n))
    rows = np.sort(_rng(15).choice(M, 40, replace=False))
    from oracle.wstack import forward_rows
    y_rows = forward_rows(n, K, omega, w, dl, stack, cen, Jr, x, rows)
    assert np.allclose(y_rows, StackedOperator(n, K, omega, w, dl, stack, cen, Jr).forward(x)[rows],
                       rtol=0, atol=1e-12 * np.abs(y_rows).max())
