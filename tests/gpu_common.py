"""Helpers shared by the GPU parity tests (inputs from ``synth``, expectations from ``oracle``)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2207_11336_gb300 as pnp  # noqa: E402


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pnp.lib()  # fails loudly when the library is missing


def to_dev_f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def to_dev_c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def to_host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def PnPError_type():
    return pnp.PnPError
