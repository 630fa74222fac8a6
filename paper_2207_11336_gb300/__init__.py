"""GB300 (sm_103a) plug-and-play forward-backward radio-interferometric imaging.

Thin Python binding over the C ABI of ``libpnp.so`` (declared in
``include/pnp.h``).  Every step of the imaging path runs in the library's CUDA
kernels; this module only marshals arguments.  PyTorch provides device memory
and streams.  Importing works without a GPU; constructing a plan needs the
built library and a CUDA device and fails loudly otherwise.

Reference: Dabbech et al. 2022, arXiv 2207.11336 (Eq. 1: y = Phi x + n,
Phi = G F Z; App. A: forward-backward; App. B/C: denoisers).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpnp.so")

PNP_W_C64, PNP_W_BF16C = 0, 1
PNP_DEN_HAAR, PNP_DEN_CNN = 0, 1
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "DIVERGED", -5: "TIMEOUT", -6: "UNSUPPORTED"}

EXPORTED = [
    "pnp_plan_create", "pnp_plan_create_stacked", "pnp_plan_destroy", "pnp_plan_get_info", "pnp_plan_set_unit_nnz",
    "pnp_plan_set_row_batch", "pnp_plan_set_holographic", "pnp_plan_export_rows", "phi_forward", "phi_adjoint", "grad_step", "op_norm",
    "pnp_den_create_haar", "pnp_den_create_cnn", "pnp_den_destroy", "denoise", "pnp_fb_run",
    "pnp_last_error", "pnp_kernel_launch_count", "pnp_plan_set_timing", "pnp_plan_read_timing",
    "pnp_plan_device_status", "pnp_haar_denoise_noalloc", "pnp_den_device_status",
    "pnp_cnn_trainer_create", "pnp_cnn_trainer_destroy", "pnp_cnn_train_step", "pnp_cnn_trainer_read",
    "pnp_cnn_num_params", "pnp_cnn_trainer_set_lr", "pnp_plan_autotune", "pnp_cnn_jacobian_norm",
    "pnp_cnn_train_step_fne", "pnp_den_create_sara", "pnp_den_sara_reweight", "pnp_sara_transform",
    "pnp_plan_create_desc", "pnp_plan_scale_data", "pnp_plan_set_compensated", "pnp_cnn_trainer_apply_update",
    "pnp_den_cnn_set_strip_rows", "pnp_den_cnn_autotune",
]
PNP_POSITIVITY_ON, PNP_POSITIVITY_OFF = 0, 1


class PnPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"PNP_ERR_{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("L", C.c_double), ("max_iter", C.c_int), ("tol", C.c_double),
                ("check_every", C.c_int), ("use_graph", C.c_int), ("diverge_factor", C.c_double),
                ("alpha", C.c_double), ("positivity", C.c_int), ("fallback", C.c_int),
                ("fallback_t", C.c_double), ("reweight_every", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("L", C.c_double), ("gamma", C.c_double),
                ("rel_change", C.c_double), ("x_norm", C.c_double), ("fallback_iter", C.c_int)]


class _PlanDesc(C.Structure):
    _fields_ = [("n", C.c_int), ("K", C.c_int), ("M", C.c_int64), ("uvw_host", C.c_void_p), ("dl", C.c_double),
                ("J_per_row_host", C.c_void_p), ("J", C.c_int), ("weight_dtype", C.c_int),
                ("block_host", C.c_void_p), ("nblocks", C.c_int), ("stack_host", C.c_void_p),
                ("nstacks", C.c_int), ("w_centres_host", C.c_void_p), ("row_scale_host", C.c_void_p),
                ("stream", C.c_void_p)]


class _Info(C.Structure):
    _fields_ = [("n", C.c_int), ("K", C.c_int), ("J", C.c_int), ("weight_dtype", C.c_int),
                ("tile", C.c_int), ("nblocks", C.c_int), ("M", C.c_int64), ("nnz", C.c_int64),
                ("n_units", C.c_int64), ("beta", C.c_double), ("dl", C.c_double),
                ("device_bytes", C.c_int64), ("region_pitch", C.c_int), ("run_max", C.c_int),
                ("unit_nnz", C.c_int64), ("row_batch", C.c_int), ("nstacks", C.c_int),
                ("holographic_bytes", C.c_int64), ("compensated", C.c_int)]


_lib = None


def lib(path: str = LIB_PATH) -> C.CDLL:
    """Load libpnp.so (built by ``paper_2207_11336_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2207_11336_gb300.build`")
    L = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    L.pnp_plan_create.argtypes = [C.POINTER(vp), i32, i32, i64, vp, dbl, vp, i32, i32, vp, i32, vp]
    L.pnp_plan_create_stacked.argtypes = [C.POINTER(vp), i32, i32, i64, vp, dbl, vp, i32, i32, vp, i32, vp, i32,
                                          vp, vp]
    L.pnp_plan_create_desc.argtypes = [C.POINTER(vp), C.POINTER(_PlanDesc)]
    L.pnp_plan_scale_data.argtypes = [vp, vp, vp]
    L.pnp_plan_set_compensated.argtypes = [vp, i32]
    L.pnp_cnn_trainer_apply_update.argtypes = [vp]
    L.pnp_den_cnn_set_strip_rows.argtypes = [vp, i32]
    L.pnp_den_cnn_autotune.argtypes = [vp, vp, i32, i32, C.POINTER(i32), C.POINTER(dbl)]
    L.pnp_plan_destroy.argtypes = [vp]
    L.pnp_plan_destroy.restype = None
    L.pnp_plan_get_info.argtypes = [vp, C.POINTER(_Info)]
    L.pnp_plan_set_unit_nnz.argtypes = [vp, i64]
    L.pnp_plan_set_row_batch.argtypes = [vp, i32]
    L.pnp_plan_set_holographic.argtypes = [vp, i32]
    L.pnp_plan_autotune.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i64), C.POINTER(dbl)]
    L.pnp_plan_export_rows.argtypes = [vp, vp, i64, vp, vp, vp]
    L.phi_forward.argtypes = [vp, vp, vp]
    L.phi_adjoint.argtypes = [vp, vp, vp]
    L.grad_step.argtypes = [vp, vp, vp, dbl, vp]
    L.op_norm.argtypes = [vp, vp, i32, dbl, C.POINTER(dbl), C.POINTER(i32)]
    L.pnp_den_create_haar.argtypes = [C.POINTER(vp), dbl, vp]
    L.pnp_den_create_cnn.argtypes = [C.POINTER(vp), vp, vp, i32, vp, i32, i32, i32, vp]
    L.pnp_den_destroy.argtypes = [vp]
    L.pnp_den_create_sara.argtypes = [C.POINTER(vp), i32, i32, dbl, dbl, i32, vp]
    L.pnp_den_sara_reweight.argtypes = [vp, vp]
    L.pnp_sara_transform.argtypes = [vp, vp, vp, i32]
    L.pnp_den_destroy.restype = None
    L.denoise.argtypes = [vp, vp, vp, i32]
    L.pnp_fb_run.argtypes = [vp, vp, vp, C.POINTER(_Params), vp, C.POINTER(_Stats)]
    L.pnp_plan_set_timing.argtypes = [vp, i32]
    L.pnp_plan_device_status.argtypes = [vp, C.POINTER(i32)]
    L.pnp_haar_denoise_noalloc.argtypes = [vp, vp, vp, i32, dbl, vp, vp]
    L.pnp_den_device_status.argtypes = [vp, C.POINTER(i32)]
    L.pnp_cnn_trainer_create.argtypes = [C.POINTER(vp), vp, i32, i32, dbl, vp]
    L.pnp_cnn_trainer_destroy.argtypes = [vp]
    L.pnp_cnn_trainer_destroy.restype = None
    L.pnp_cnn_train_step.argtypes = [vp, vp, vp, dbl, i32, C.POINTER(dbl)]
    L.pnp_cnn_trainer_read.argtypes = [vp, vp, vp, i32]
    L.pnp_cnn_num_params.restype = i64
    L.pnp_cnn_trainer_set_lr.argtypes = [vp, dbl]
    L.pnp_cnn_jacobian_norm.argtypes = [vp, vp, vp, i32, vp, vp]
    L.pnp_cnn_train_step_fne.argtypes = [vp, vp, vp, dbl, vp, i32, dbl, dbl, i32, C.POINTER(dbl), C.POINTER(dbl)]
    L.pnp_plan_read_timing.argtypes = [vp, vp, vp]
    L.pnp_last_error.restype = C.c_char_p
    L.pnp_kernel_launch_count.restype = i64
    for name in ("pnp_plan_create", "pnp_plan_create_stacked", "pnp_plan_get_info", "pnp_plan_set_unit_nnz",
                 "pnp_plan_set_row_batch", "pnp_plan_set_holographic",
                 "pnp_plan_export_rows",
                 "phi_forward", "phi_adjoint", "grad_step", "op_norm", "pnp_den_create_haar",
                 "pnp_den_create_cnn", "denoise", "pnp_fb_run", "pnp_plan_set_timing",
                 "pnp_plan_read_timing", "pnp_plan_device_status", "pnp_haar_denoise_noalloc",
                 "pnp_den_device_status", "pnp_cnn_trainer_create", "pnp_cnn_train_step",
                 "pnp_cnn_trainer_read", "pnp_cnn_trainer_set_lr", "pnp_plan_autotune", "pnp_cnn_jacobian_norm",
                 "pnp_cnn_train_step_fne", "pnp_den_create_sara", "pnp_den_sara_reweight",
                 "pnp_sara_transform", "pnp_plan_create_desc", "pnp_plan_scale_data",
                 "pnp_plan_set_compensated", "pnp_cnn_trainer_apply_update", "pnp_den_cnn_set_strip_rows",
                 "pnp_den_cnn_autotune"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise PnPError(rc, lib().pnp_last_error().decode())


def kernel_launches() -> int:
    """Number of this library's kernels launched in this process."""
    return int(lib().pnp_kernel_launch_count())


def _ptr(t) -> int:
    return t.data_ptr()


def _cuda_f32(t, shape, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA float32 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _cuda_c64(t, m, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA complex64 tensor")
    if t.numel() != m:
        raise ValueError(f"{name} has {t.numel()} entries, expected {m}")
    return t


def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


@dataclass
class FBStats:
    iters: int
    L: float
    gamma: float
    rel_change: float
    x_norm: float
    fallback_iter: int = -1


class Plan:
    """Measurement operator Phi = G F Z (Eq. 1) with w-terms folded into G (App. E).

    ``omega``: (M, 2) float64 rad/pixel (column 0 pairs with image axis 0);
    ``w``: (M,) wavelengths; ``dl``: pixel size [rad] for the w-term (0: none);
    ``J_per_row``: (M,) int8 supports in [J, 16] or None;
    ``stack``, ``w_centres``: the w-stacking hybrid of App. E (Eq. phip): (M,) int32
    stack ids in [0, P) and the P stack centres [wavelengths]; Z_p then carries the
    centre chirp and the rows of G only the offset w - w_p.
    """

    def __init__(self, n, K, omega, w=None, dl=0.0, J_per_row=None, J=7, weight_dtype="c64",
                 block=None, nblocks=1, stream=None, stack=None, w_centres=None, row_scale=None):
        import torch
        L = lib()
        omega = np.asarray(omega, dtype=np.float64)
        M = omega.shape[0]
        uvw = np.zeros((M, 3), dtype=np.float64)
        uvw[:, :2] = omega
        if w is not None:
            uvw[:, 2] = np.asarray(w, dtype=np.float64)
        uvw = np.ascontiguousarray(uvw)
        jr = None if J_per_row is None else np.ascontiguousarray(J_per_row, dtype=np.int8)
        blk = None if block is None else np.ascontiguousarray(block, dtype=np.int32)
        wc = None if w_centres is None else np.ascontiguousarray(w_centres, dtype=np.float64)
        stk = None if wc is None else np.ascontiguousarray(np.zeros(M) if stack is None else stack, dtype=np.int32)
        rs = None if row_scale is None else np.ascontiguousarray(row_scale, dtype=np.float64)
        if rs is not None and rs.shape != (M,):
            raise ValueError(f"row_scale has shape {rs.shape}, expected ({M},)")
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self._h = C.c_void_p()
        wd = PNP_W_BF16C if weight_dtype in ("bf16", PNP_W_BF16C) else PNP_W_C64
        ptr = lambda a: None if a is None else a.ctypes.data  # noqa: E731
        desc = _PlanDesc(int(n), int(K), int(M), uvw.ctypes.data, float(dl), ptr(jr), int(J), wd, ptr(blk),
                         int(nblocks), ptr(stk), 1 if wc is None else int(wc.size), ptr(wc), ptr(rs),
                         _stream_handle(self.stream).value)
        _check(L.pnp_plan_create_desc(C.byref(self._h), C.byref(desc)))
        self.weighted = rs is not None
        self.n, self.K, self.M = int(n), int(K), int(M)

    # ------------------------------------------------------------------ info
    @property
    def info(self) -> dict:
        inf = _Info()
        _check(lib().pnp_plan_get_info(self._h, C.byref(inf)))
        return {f: getattr(inf, f) for f, _ in _Info._fields_}

    def set_unit_nnz(self, unit_nnz: int):
        _check(lib().pnp_plan_set_unit_nnz(self._h, int(unit_nnz)))

    def set_holographic(self, enable: bool = True):
        """Use the holographic H = G^H G in the FB loop and op_norm (App. E, Eq. phidagphi)."""
        _check(lib().pnp_plan_set_holographic(self._h, 1 if enable else 0))

    def set_compensated(self, enable: bool = True):
        """Compensated (TwoSum) summation of the gridding pass's flushes into the output grid."""
        _check(lib().pnp_plan_set_compensated(self._h, 1 if enable else 0))

    def set_row_batch(self, row_batch: int):
        """Rows of a run whose residuals one warp forms together (1, 2 or 4)."""
        _check(lib().pnp_plan_set_row_batch(self._h, int(row_batch)))

    def autotune(self, reps: int = 2) -> dict:
        """Time the gridding pass's run cap x unit size x row batch candidates and keep the fastest."""
        r, u, ms = C.c_int(), C.c_int64(), C.c_double()
        _check(lib().pnp_plan_autotune(self._h, int(reps), C.byref(r), C.byref(u), C.byref(ms)))
        return {"run_max": r.value, "unit_nnz": u.value, "row_batch": self.info["row_batch"],
                "gridding_ms": ms.value}

    def device_status(self) -> int:
        """Device status flags (0 when every kernel check passed)."""
        f = C.c_int()
        _check(lib().pnp_plan_device_status(self._h, C.byref(f)))
        return f.value

    def set_timing(self, enable: bool):
        """Bracket each eager FFT / gridding stage with CUDA events."""
        _check(lib().pnp_plan_set_timing(self._h, 1 if enable else 0))

    def read_timing(self):
        """{stage: (total ms, launches)} for 'fft_forward', 'gridding', 'fft_adjoint'; clears the record."""
        ms = np.zeros(3, dtype=np.float64)
        cnt = np.zeros(3, dtype=np.int64)
        _check(lib().pnp_plan_read_timing(self._h, ms.ctypes.data, cnt.ctypes.data))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(("fft_forward", "gridding", "fft_adjoint"))}

    def export_rows(self, rows):
        """(offsets, weights complex64, canonical columns k0*K + k1) of the given rows of G."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        off = np.zeros(rows.size + 1, dtype=np.int64)
        _check(lib().pnp_plan_export_rows(self._h, rows.ctypes.data, rows.size, off.ctypes.data, None, None))
        wts = np.zeros(int(off[-1]), dtype=np.complex64)
        cols = np.zeros(int(off[-1]), dtype=np.int32)
        _check(lib().pnp_plan_export_rows(self._h, rows.ctypes.data, rows.size, off.ctypes.data,
                                          wts.ctypes.data, cols.ctypes.data))
        return off, wts, cols

    # ------------------------------------------------------------------ operator
    def scale_data(self, y, out=None):
        """D y for the plan's data weights D (a copy without weights): the weighted data."""
        import torch
        _cuda_c64(y, self.M, "y")
        o = torch.empty_like(y) if out is None else out
        _cuda_c64(o, self.M, "out")
        _check(lib().pnp_plan_scale_data(self._h, _ptr(y), _ptr(o)))
        return o

    def phi_forward(self, x, out=None):
        """y = Phi x (Eq. 1)."""
        import torch
        _cuda_f32(x, (self.n, self.n), "x")
        y = torch.empty(self.M, dtype=torch.complex64, device=x.device) if out is None else out
        _cuda_c64(y, self.M, "y")
        _check(lib().phi_forward(self._h, _ptr(x), _ptr(y)))
        return y

    def phi_adjoint(self, y, out=None):
        """x = Re{Phi^H y} (App. A)."""
        import torch
        _cuda_c64(y, self.M, "y")
        x = torch.empty((self.n, self.n), dtype=torch.float32, device=y.device) if out is None else out
        _cuda_f32(x, (self.n, self.n), "out")
        _check(lib().phi_adjoint(self._h, _ptr(y), _ptr(x)))
        return x

    def grad_step(self, x, y, gamma, out=None):
        """x - gamma Re{Phi^H (Phi x - y)} (forward step of Eq. fb)."""
        import torch
        _cuda_f32(x, (self.n, self.n), "x")
        _cuda_c64(y, self.M, "y")
        o = torch.empty_like(x) if out is None else out
        _cuda_f32(o, (self.n, self.n), "out")
        _check(lib().grad_step(self._h, _ptr(x), _ptr(y), float(gamma), _ptr(o)))
        return o

    def op_norm(self, v0=None, max_it=1000, tol=1e-7):
        """(L, iterations): ||Re{Phi^H Phi}||_S by power iteration (App. A)."""
        if v0 is not None:
            _cuda_f32(v0, (self.n, self.n), "v0")
        Lv = C.c_double()
        it = C.c_int()
        _check(lib().op_norm(self._h, None if v0 is None else _ptr(v0), int(max_it), float(tol),
                             C.byref(Lv), C.byref(it)))
        return Lv.value, it.value

    def fb_run(self, den, y, x0=None, gamma=0.0, L=0.0, max_iter=200, tol=0.0, check_every=10,
               use_graph=True, diverge_factor=0.0, inplace=False, alpha=1.0, positivity=True,
               fallback_t=None, reweight_every=0):
        """Run Eq. fb with denoiser ``den`` from x0 (zeros if None); returns (x, FBStats).

        ``alpha`` rescales the problem as in App. C (Eq. invpb2): the loop iterates on y / alpha
        from x0 / alpha and returns alpha x.  ``positivity`` keeps the final max(0, .) of the
        denoiser.  ``fallback_t`` (learned denoiser only): on divergence, continue from the last
        checked finite iterate with the Haar denoiser at this threshold (rescaled units).
        ``reweight_every`` (SARA denoiser only): re-form the uSARA weights from the iterate every this
        many iterations.  With ``inplace`` the iterate is updated in x0 itself."""
        import torch
        _cuda_c64(y, self.M, "y")
        if x0 is None:
            x = torch.zeros((self.n, self.n), dtype=torch.float32, device=y.device)
        else:
            x = x0 if inplace else x0.clone()
        _cuda_f32(x, (self.n, self.n), "x0")
        prm = _Params(float(gamma), float(L), int(max_iter), float(tol), int(check_every),
                      1 if use_graph else 0, float(diverge_factor), float(alpha),
                      PNP_POSITIVITY_ON if positivity else PNP_POSITIVITY_OFF,
                      0 if fallback_t is None else 1, 0.0 if fallback_t is None else float(fallback_t),
                      int(reweight_every))
        st = _Stats()
        _check(lib().pnp_fb_run(self._h, den._h, _ptr(y), C.byref(prm), _ptr(x), C.byref(st)))
        return x, FBStats(st.iters, st.L, st.gamma, st.rel_change, st.x_norm, st.fallback_iter)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().pnp_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Denoiser:
    _h = None

    def denoise(self, x, out=None):
        """x_out = D(x)."""
        import torch
        n = x.shape[0]
        _cuda_f32(x, (n, n), "x")
        o = torch.empty_like(x) if out is None else out
        _check(lib().denoise(self._h, _ptr(x), _ptr(o), int(n)))
        return o

    def device_status(self) -> int:
        """Device status flags of this denoiser's kernels (0 when every check passed)."""
        f = C.c_int()
        _check(lib().pnp_den_device_status(self._h, C.byref(f)))
        return f.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().pnp_den_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HaarDenoiser(_Denoiser):
    """Haar soft-threshold at t + positivity (App. B; t = tau / sqrt(2L), Eq. lambda)."""

    def __init__(self, t: float, stream=None):
        lib()
        self._h = C.c_void_p()
        _check(lib().pnp_den_create_haar(C.byref(self._h), float(t), _stream_handle(stream)))
        self.t = float(t)


class SaraDenoiser(_Denoiser):
    """uSARA's denoiser (App. B): the prox of gamma_lambda ||W Psi^T x||_1 + positivity for the SARA
    dictionary by ``prox_iters`` dual forward-backward iterations (warm-started); ``reweight(x)``
    sets W from the log-sum prior at x."""

    def __init__(self, n: int, gamma_lambda: float, rho: float, prox_iters: int = 20, levels: int = 4,
                 stream=None):
        lib()
        self.n = int(n)
        self._h = C.c_void_p()
        _check(lib().pnp_den_create_sara(C.byref(self._h), self.n, int(levels), float(gamma_lambda), float(rho),
                                         int(prox_iters), _stream_handle(stream)))

    def reweight(self, x):
        _cuda_f32(x, (self.n, self.n), "x")
        _check(lib().pnp_den_sara_reweight(self._h, _ptr(x)))

    def analysis(self, x):
        """Psi^T x: (9, n, n)."""
        import torch
        _cuda_f32(x, (self.n, self.n), "x")
        out = torch.empty((9, self.n, self.n), dtype=torch.float32, device=x.device)
        _check(lib().pnp_sara_transform(self._h, _ptr(x), _ptr(out), 1))
        return out

    def synthesis(self, c):
        """Psi c for c of shape (9, n, n)."""
        import torch
        _cuda_f32(c, (9, self.n, self.n), "c")
        out = torch.empty((self.n, self.n), dtype=torch.float32, device=c.device)
        _check(lib().pnp_sara_transform(self._h, _ptr(c), _ptr(out), -1))
        return out


def pack_cnn_weights(params) -> np.ndarray:
    """Flatten [(W (co, ci, 3, 3), b (co,)), ...] into the float32 layout of pnp_den_create_cnn."""
    return np.ascontiguousarray(np.concatenate([np.concatenate([np.ravel(W), np.ravel(b)])
                                                for W, b in params]).astype(np.float32))


def unpack_cnn_weights(flat, channels=64, depth=8):
    """Inverse of ``pack_cnn_weights``: flat float array -> [(W, b), ...] (float64)."""
    flat = np.asarray(flat, dtype=np.float64)
    shapes = [(channels, 1)] + [(channels, channels)] * (depth - 2) + [(1, channels)]
    out, off = [], 0
    for co, ci in shapes:
        W = flat[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        out.append((W.copy(), flat[off:off + co].copy()))
        off += co
    return out


class CnnTrainer:
    """Adam training of the residual CNN on batches of size x size images (App. C)."""

    def __init__(self, params, batch: int, size: int, lr: float = 1e-4, stream=None):
        lib()
        self.batch, self.size = int(batch), int(size)
        self._h = C.c_void_p()
        w = pack_cnn_weights(params)
        if w.size != lib().pnp_cnn_num_params():
            raise ValueError("parameters do not match the 8-layer 64-channel network")
        _check(lib().pnp_cnn_trainer_create(C.byref(self._h), w.ctypes.data, self.batch, self.size,
                                            float(lr), _stream_handle(stream)))

    def step(self, u, noise, sigma: float, update: bool = True, want_loss: bool = False):
        """One training step on device batches u, noise (batch x size x size float32)."""
        shape = (self.batch, self.size, self.size)
        _cuda_f32(u, shape, "u")
        _cuda_f32(noise, shape, "noise")
        loss = C.c_double(0.0)
        _check(lib().pnp_cnn_train_step(self._h, _ptr(u), _ptr(noise), float(sigma), 1 if update else 0,
                                        C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def apply_update(self):
        """One Adam step on the gradients accumulated by steps with update=False (clears them)."""
        _check(lib().pnp_cnn_trainer_apply_update(self._h))

    def set_lr(self, lr: float):
        """Adam step size for the following steps (moments are kept)."""
        _check(lib().pnp_cnn_trainer_set_lr(self._h, float(lr)))

    def step_fne(self, u, noise, sigma: float, v0, iters: int, lam: float, eps: float = 0.0,
                 update: bool = True, want_values: bool = False):
        """One training step with the soft firm non-expansiveness penalty (Eq. training_loss):
        l1 loss + lam/B sum_b max(||J_Q v_b||^2, 1 - eps), v_b from ``iters`` power iterations
        from v0.  Returns (loss, penalty) when ``want_values``."""
        shape = (self.batch, self.size, self.size)
        _cuda_f32(u, shape, "u")
        _cuda_f32(noise, shape, "noise")
        _cuda_f32(v0, shape, "v0")
        loss, pen = C.c_double(0.0), C.c_double(0.0)
        _check(lib().pnp_cnn_train_step_fne(self._h, _ptr(u), _ptr(noise), float(sigma), _ptr(v0), int(iters),
                                            float(lam), float(eps), 1 if update else 0,
                                            C.byref(loss) if want_values else None,
                                            C.byref(pen) if want_values else None))
        return (loss.value, pen.value) if want_values else None

    def jacobian_norm(self, z, v0, iters: int = 20):
        """(sigma per image, last unit iterate): ||grad (2D - I)(z)||_S by power iteration, the
        quantity the firm non-expansiveness constraint of Eq. training_loss bounds by 1."""
        import torch
        shape = (self.batch, self.size, self.size)
        _cuda_f32(z, shape, "z")
        _cuda_f32(v0, shape, "v0")
        sig = np.zeros(self.batch, dtype=np.float64)
        v = torch.empty(shape, dtype=torch.float32, device=z.device)
        _check(lib().pnp_cnn_jacobian_norm(self._h, _ptr(z), _ptr(v0), int(iters), sig.ctypes.data, _ptr(v)))
        return sig, v

    def read(self, weights=True, grads=False, clear_grads=False):
        """(params or None, flat gradients or None) from the device."""
        n = int(lib().pnp_cnn_num_params())
        w = np.zeros(n, dtype=np.float32) if weights else None
        g = np.zeros(n, dtype=np.float32) if grads else None
        _check(lib().pnp_cnn_trainer_read(self._h, None if w is None else w.ctypes.data,
                                          None if g is None else g.ctypes.data, 1 if clear_grads else 0))
        return (unpack_cnn_weights(w) if w is not None else None), g

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().pnp_cnn_trainer_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CnnDenoiser(_Denoiser):
    """Residual CNN denoiser D(z) = max(0, z - N(z)) (App. C), faceted with a halo (App. D)."""

    def __init__(self, params, n: int, facet_rows=None, facet_cols=None, halo: int = 32, stream=None):
        lib()
        wts = pack_cnn_weights(params)
        fr = None if facet_rows is None else np.ascontiguousarray(facet_rows, dtype=np.int32)
        fc = None if facet_cols is None else np.ascontiguousarray(facet_cols, dtype=np.int32)
        self._h = C.c_void_p()
        _check(lib().pnp_den_create_cnn(C.byref(self._h), wts.ctypes.data,
                                        None if fr is None else fr.ctypes.data, 0 if fr is None else fr.size,
                                        None if fc is None else fc.ctypes.data, 0 if fc is None else fc.size,
                                        int(halo), int(n), _stream_handle(stream)))
        self.n = int(n)

    def set_strip_rows(self, rows: int):
        """Output rows per convolution work strip (a performance setting; results are unchanged)."""
        _check(lib().pnp_den_cnn_set_strip_rows(self._h, int(rows)))

    def autotune(self, z, reps: int = 3) -> dict:
        """Time the denoise of the device image z for each strip height and keep the fastest."""
        _cuda_f32(z, (self.n, self.n), "z")
        rows, ms = C.c_int(), C.c_double()
        _check(lib().pnp_den_cnn_autotune(self._h, _ptr(z), self.n, int(reps), C.byref(rows), C.byref(ms)))
        return {"strip_rows": rows.value, "denoise_ms": ms.value}


def haar_denoise_noalloc(z, t: float, x_prev=None, out=None, norms=None, stream=None):
    """Haar denoiser + FP64 norms through the allocation-free entry point.

    For callers that cannot let the library allocate: every buffer is passed
    in (``out`` n x n float32 and ``norms`` 2 float64 on the device are
    created here only when omitted).  Returns (out, norms) with
    norms = (||out - x_prev||^2, ||out||^2).
    """
    import torch
    n = z.shape[0]
    _cuda_f32(z, (n, n), "z")
    if x_prev is not None:
        _cuda_f32(x_prev, (n, n), "x_prev")
    o = torch.empty_like(z) if out is None else out
    nr = torch.empty(2, dtype=torch.float64, device=z.device) if norms is None else norms
    _check(lib().pnp_haar_denoise_noalloc(_ptr(z), None if x_prev is None else _ptr(x_prev), _ptr(o),
                                          int(n), float(t), _ptr(nr), _stream_handle(stream)))
    return o, nr
