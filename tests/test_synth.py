"""Checks of the seeded synthetic input generators (no method arithmetic)."""
import numpy as np

import synth


def test_noise_has_unit_power_and_is_seeded():
    a = synth.complex_normal(200_000, synth.rng_for("noise"))
    b = synth.complex_normal(200_000, synth.rng_for("noise"))
    assert np.array_equal(a, b)
    assert abs(np.mean(np.abs(a) ** 2) - 1.0) < 0.01


def test_uv_geometry_and_supports():
    p = synth.make_problem("C1", M=50_000, n=64, K=128)
    r = np.hypot(p["omega"][:, 0], p["omega"][:, 1])
    assert abs(r.max() - 0.8 * np.pi) < 1e-12
    Jr = p["J_per_row"]
    assert set(np.unique(Jr)) == {7, 9, 12, 16}
    aw = np.abs(p["w"])
    assert aw[Jr == 7].max() <= aw[Jr == 16].min()
    assert np.max(aw) * p["dl"] ** 2 * 64 * 128 == 4.0 or abs(np.max(aw) * p["dl"] ** 2 * 64 * 128 - 4.0) < 1e-9


def test_blocks_and_facets():
    p = synth.make_problem("C3", M=2_000_000, n=512, K=1024)
    cnt = np.bincount(p["block"], minlength=64)
    assert cnt.sum() == 2_000_000 and (cnt > 0).all()
    assert p["facet_rows"].sum() == 512 and p["facet_cols"].sum() == 512
    assert len(p["facet_rows"]) == 4


def test_sky_nonnegative_and_training_normalised():
    x = synth.sky_model(64, synth.rng_for("sky"))
    assert x.min() >= 0 and x.max() > 0
    t = synth.training_image(64, synth.rng_for("train"))
    assert t.max() == 1.0 and t.min() >= 0


def test_briggs_weights_limits_and_robust_zero():
    """Briggs weights (Sec. 3, robust 0): natural weighting for large robust, uniform weighting (the
    summed weight of every occupied uv cell equal) for very negative robust, and the formula
    1 / (1 + W_k f^2) on a hand-counted case."""
    rng = np.random.default_rng(5)
    n = 16
    omega = rng.uniform(-0.9 * np.pi, 0.9 * np.pi, (400, 2))
    assert np.allclose(synth.briggs_weights(omega, n, 8.0), 1.0, atol=1e-10)
    wu = synth.briggs_weights(omega, n, -8.0)
    k = np.rint(omega * n / (2 * np.pi)).astype(int) % n
    cell, conj = k[:, 0] * n + k[:, 1], ((-k[:, 0]) % n) * n + ((-k[:, 1]) % n)
    W = np.bincount(cell, minlength=n * n) + np.bincount(conj, minlength=n * n)
    per_cell = np.bincount(cell, weights=wu, minlength=n * n) + np.bincount(conj, weights=wu, minlength=n * n)
    occ = W > 0
    assert np.allclose(per_cell[occ], per_cell[occ][0], rtol=1e-6)   # flat summed density
    # three rows: two in one cell, one alone (no conjugate overlap at these cells)
    om = np.array([[3.2, 1.1], [2.9, 0.8], [-5.1, 6.0]]) * (2 * np.pi / n)
    wb = synth.briggs_weights(om, n, 0.0)
    Wk = np.array([2.0, 2.0, 1.0])
    f2 = 25.0 / (Wk.sum() / 3.0)
    assert np.allclose(wb, 1.0 / (1.0 + Wk * f2), rtol=1e-14)
