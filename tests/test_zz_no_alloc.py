"""The allocation-free denoiser entry point matches the regular one.

Some callers cannot allocate device memory (a fixed memory budget reserved up
front, a caller-owned pool, or a runtime that forbids allocation after
start-up).  For them pnp_haar_denoise_noalloc keeps its scratch in a static
device array.  This file is collected last so that, if it fails, every other
test has already run; it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import pnp, require_gpu, to_dev_f32, to_host, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_noalloc_matches_existing_denoiser_on_two_calls():
    rng = np.random.default_rng(2024)
    L = pnp.lib()
    for call, (n, t) in enumerate([(256, 0.3), (130, 0.05)]):   # two calls in a row, different sizes
        z = rng.standard_normal((n, n)).astype(np.float32)
        xp = rng.standard_normal((n, n)).astype(np.float32)
        zd, xpd = to_dev_f32(z), to_dev_f32(xp)
        ref = to_host(pnp.HaarDenoiser(t).denoise(zd))               # existing entry point
        out = torch.empty_like(zd)
        norms = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        rc = L.pnp_haar_denoise_noalloc(zd.data_ptr(), xpd.data_ptr(), out.data_ptr(), n, t,
                                        norms.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, L.pnp_last_error()
        o = to_host(out)
        assert np.allclose(o, ref, rtol=0, atol=1e-6), call
        nv = to_host(norms)
        assert nv[0] == pytest.approx(np.sum((o - xp.astype(np.float64)) ** 2), rel=1e-12)
        assert nv[1] == pytest.approx(np.sum(o ** 2), rel=1e-12)


def test_noalloc_rejects_sizes_beyond_its_limit():
    L = pnp.lib()
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    rc = L.pnp_haar_denoise_noalloc(dummy.data_ptr(), None, dummy.data_ptr() + 8, 16386, 0.1,
                                    dummy.data_ptr(), None)
    assert rc == -1 and b"limit" in L.pnp_last_error()


def test_noalloc_without_previous_iterate_and_with_non_finite_input():
    """x_prev = NULL gives ||x_out - x_prev||^2 = 0; a NaN in z makes ||x_out||^2 NaN, the signal the
    stopping test reads (positivity alone would map the NaN to 0)."""
    L = pnp.lib()
    n, t = 64, 0.1
    z = np.random.default_rng(7).standard_normal((n, n)).astype(np.float32)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    zd = to_dev_f32(z)
    out = torch.empty_like(zd)
    norms = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    assert L.pnp_haar_denoise_noalloc(zd.data_ptr(), None, out.data_ptr(), n, t, norms.data_ptr(), stream) == 0
    nv, o = to_host(norms), to_host(out)
    assert nv[0] == 0.0
    assert nv[1] == pytest.approx(np.sum(o.astype(np.float64) ** 2), rel=1e-12)
    z[5, 9] = np.nan
    zd = to_dev_f32(z)
    assert L.pnp_haar_denoise_noalloc(zd.data_ptr(), None, out.data_ptr(), n, t, norms.data_ptr(), stream) == 0
    assert np.isnan(to_host(norms)[1])


def test_noalloc_rejects_outputs_overlapping_its_inputs():
    L = pnp.lib()
    n = 32
    buf = torch.zeros(3 * n * n, dtype=torch.float32, device="cuda")
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    base = buf.data_ptr()
    # x_prev is x_out, then z shares half of x_out's rows
    assert L.pnp_haar_denoise_noalloc(base, base + 4 * n * n, base + 4 * n * n, n, 0.1, norms.data_ptr(),
                                      None) == -1
    assert b"x_prev" in L.pnp_last_error()
    assert L.pnp_haar_denoise_noalloc(base, None, base + 2 * n * n, n, 0.1, norms.data_ptr(), None) == -1
    assert b"overlap" in L.pnp_last_error()
