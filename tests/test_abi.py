"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every declared symbol."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pnp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


@pytest.fixture(scope="module")
def libpath():
    from paper_2207_11336_gb300 import LIB_PATH
    from paper_2207_11336_gb300 import build as b
    if not os.path.exists(LIB_PATH):
        b.build()
    return LIB_PATH


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("phi_forward", "phi_adjoint", "grad_step", "op_norm", "denoise", "pnp_fb_run",
                 "pnp_plan_create", "pnp_den_create_haar", "pnp_den_create_cnn", "pnp_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(declared_functions()) <= exported


def test_binding_names_match_header():
    import paper_2207_11336_gb300 as pnp
    assert set(pnp.EXPORTED) == set(declared_functions())


def test_error_path_without_gpu(libpath):
    import paper_2207_11336_gb300 as pnp
    L = pnp.lib(libpath)
    h = ctypes.c_void_p()
    rc = L.pnp_plan_create(ctypes.byref(h), 15, 64, 0, None, 0.0, None, 7, 0, None, 1, None)
    assert rc == -1 and b"even" in L.pnp_last_error()
    rc = L.pnp_den_create_haar(ctypes.byref(h), -1.0, None)
    assert rc == -1


def test_argument_checks_of_the_newer_entry_points_without_gpu(libpath):
    """Every check below returns before any CUDA call, so it runs on a machine without a GPU."""
    import paper_2207_11336_gb300 as pnp
    L = pnp.lib(libpath)
    h = ctypes.c_void_p()
    uvw = (ctypes.c_double * 3)(0.1, 0.2, 1.0)
    stk = (ctypes.c_int32 * 1)(0)
    cen = (ctypes.c_double * 2)(0.0, 1.0)
    # w-stacked plans: stack count, missing centres, no w-term
    rc = L.pnp_plan_create_stacked(ctypes.byref(h), 16, 64, 1, uvw, 0.01, None, 7, 0, None, 1, stk, 0, cen, None)
    assert rc == -1 and b"nstacks" in L.pnp_last_error()
    rc = L.pnp_plan_create_stacked(ctypes.byref(h), 16, 64, 1, uvw, 0.01, None, 7, 0, None, 1, stk, 2, None, None)
    assert rc == -1 and b"w_centres" in L.pnp_last_error()
    rc = L.pnp_plan_create_stacked(ctypes.byref(h), 16, 64, 1, uvw, 0.0, None, 7, 0, None, 1, stk, 2, cen, None)
    assert rc == -1 and b"dl" in L.pnp_last_error()
    # SARA denoiser: levels and image side
    rc = L.pnp_den_create_sara(ctypes.byref(h), 24, 4, 0.1, 0.1, 5, None)
    assert rc == -1 and b"2^levels" in L.pnp_last_error()
    rc = L.pnp_den_create_sara(ctypes.byref(h), 64, 0, 0.1, 0.1, 5, None)
    assert rc == -1
    rc = L.pnp_den_create_sara(ctypes.byref(h), 64, 4, 0.1, 0.0, 5, None)
    assert rc == -1 and b"SARA" in L.pnp_last_error()
    # NULL handles
    assert L.pnp_plan_set_holographic(None, 1) == -1
    assert L.pnp_plan_set_row_batch(None, 2) == -1
    assert L.pnp_den_sara_reweight(None, None) == -1
    assert L.pnp_sara_transform(None, None, None, 1) == -1
    sig = (ctypes.c_double * 1)()
    assert L.pnp_cnn_jacobian_norm(None, None, None, 1, sig, None) == -1
    assert L.pnp_cnn_train_step_fne(None, None, None, 0.1, None, 1, 1.0, 0.05, 1, None, None) == -1
