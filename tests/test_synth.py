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
