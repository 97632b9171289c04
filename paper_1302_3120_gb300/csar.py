"""Thin ctypes binding of libcsar (include/csar.h) with the same entry-point names.

Argument marshalling only: every step of the imaging path runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current stream.  The
library must have been built (``paper_1302_3120_gb300.build.build()``); when it is
missing the import of this module raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CSAR_LIB_PATH selects another build of the library (the checked build,
# libcsar_checked.so); by default the in-tree libcsar.so
LIB_PATH = os.environ.get("CSAR_LIB_PATH") or os.path.join(_HERE, "libcsar.so")

CSAR_OK = 0
STATUS_NAMES = {0: "CSAR_OK", 1: "CSAR_E_INVALID", 2: "CSAR_E_UNSUPPORTED", 3: "CSAR_E_OOM",
                4: "CSAR_E_CUDA", 5: "CSAR_E_TIMEOUT", 6: "CSAR_E_NONFINITE", 7: "CSAR_E_INTERNAL"}
MU_MODES = {"fixed": 0, "niht": 1}
THRESH = {"soft": 0, "half": 1, "hard": 2}
N_PASSES = 6
PASS_NAMES = ("C1_sparse_fft", "R1_range_G", "C2_residue", "R2_range_M", "C3_select", "select_threshold")


class CsarError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("n_az", ctypes.c_int32), ("n_rg", ctypes.c_int32),
                ("wavelength", ctypes.c_double), ("velocity", ctypes.c_double),
                ("r0", ctypes.c_double), ("prf", ctypes.c_double),
                ("bandwidth", ctypes.c_double), ("pulse_len", ctypes.c_double),
                ("fs", ctypes.c_double), ("antenna_len", ctypes.c_double),
                ("c", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("iters", ctypes.c_int32), ("mu_mode", ctypes.c_int32),
                ("mu", ctypes.c_float), ("thresh", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("resid_sq", ctypes.POINTER(ctypes.c_double)),
                ("mu", ctypes.POINTER(ctypes.c_float)),
                ("sigma", ctypes.POINTER(ctypes.c_float)),
                ("nnz", ctypes.POINTER(ctypes.c_int64))]


EXPORTS = ("csar_plan_create", "csar_plan_destroy", "csar_G", "csar_M", "csar_ita_step",
           "csar_solve", "csar_solve_host", "csar_solve_profile", "csar_plan_check",
           "csar_last_error", "csar_version", "csar_af_solve", "csar_af_loss", "csar_af_backward",
           "csar_G_noalloc", "csar_batch_create", "csar_batch_destroy", "csar_solve_batched",
           "csar_batch_check", "csar_autotune", "csar_selftest_wait_timeout", "csar_echo_points",
           "csar_debug_selection_enable", "csar_debug_selection_read", "csar_plan_set_pulse",
           "csar_debug_fail_alloc")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcsar is not built ({LIB_PATH} missing); run "
                          "paper_1302_3120_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32
    lib.csar_plan_create.argtypes = [ctypes.POINTER(Params), u32, ctypes.POINTER(vp)]
    lib.csar_plan_destroy.argtypes = [vp]
    lib.csar_G.argtypes = [vp, vp, vp, vp]
    lib.csar_M.argtypes = [vp, vp, vp, vp]
    lib.csar_ita_step.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Opts), vp, vp]
    lib.csar_solve.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(Stats), vp]
    lib.csar_solve_host.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(Stats), vp]
    lib.csar_solve_profile.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Opts),
                                       ctypes.POINTER(ctypes.c_float), i32, vp]
    lib.csar_plan_check.argtypes = [vp]
    lib.csar_af_solve.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(Opts), i32, vp]
    lib.csar_af_loss.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.csar_af_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.csar_G_noalloc.argtypes = [ctypes.POINTER(Params), vp, vp, vp]
    lib.csar_batch_create.argtypes = [ctypes.POINTER(Params), i32, u32, ctypes.POINTER(vp)]
    lib.csar_batch_destroy.argtypes = [vp]
    lib.csar_solve_batched.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(Opts), vp]
    lib.csar_batch_check.argtypes = [vp]
    lib.csar_autotune.argtypes = [ctypes.POINTER(Params), i32, ctypes.POINTER(i32)]
    lib.csar_selftest_wait_timeout.argtypes = [i32]
    lib.csar_echo_points.argtypes = [ctypes.POINTER(Params), vp, vp, vp, ctypes.c_int64, vp, i32, vp]
    lib.csar_plan_set_pulse.argtypes = [vp, vp]
    lib.csar_debug_fail_alloc.argtypes = [i32]
    lib.csar_debug_selection_enable.argtypes = [vp, ctypes.c_int64]
    lib.csar_debug_selection_read.argtypes = [vp, vp, vp, vp, ctypes.c_int64,
                                              ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(u32),
                                              ctypes.POINTER(ctypes.c_float),
                                              ctypes.POINTER(ctypes.c_float)]
    lib.csar_last_error.restype = ctypes.c_char_p
    lib.csar_version.restype = i32
    for name in ("csar_plan_create", "csar_plan_destroy", "csar_G", "csar_M", "csar_ita_step",
                 "csar_solve", "csar_solve_host", "csar_solve_profile", "csar_plan_check",
                 "csar_af_solve", "csar_af_loss", "csar_af_backward", "csar_G_noalloc",
                 "csar_batch_create", "csar_batch_destroy", "csar_solve_batched", "csar_batch_check",
                 "csar_autotune", "csar_echo_points", "csar_debug_selection_enable",
                 "csar_debug_selection_read", "csar_plan_set_pulse", "csar_debug_fail_alloc"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


def _check(st: int, where: str) -> None:
    if st != CSAR_OK:
        raise CsarError(st, where, lib.csar_last_error().decode())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, n: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise TypeError(f"{name}: need contiguous {dtype} with {n} elements, got {t.dtype} "
                        f"{tuple(t.shape)}")


def params_of(g) -> Params:
    """csar_params from any object with the system-parameter attributes."""
    return Params(int(g.n_az), int(g.n_rg), float(g.wavelength), float(g.velocity), float(g.r0),
                  float(g.prf), float(g.bandwidth), float(g.pulse_len), float(g.fs),
                  float(getattr(g, "antenna_len", 0.0)), float(getattr(g, "c", 0.0)))


class Plan:
    """Owns a csar_plan handle (destroyed with the object)."""

    def __init__(self, handle: int, n_az: int, n_rg: int):
        self.handle = ctypes.c_void_p(handle)
        self.n_az, self.n_rg = n_az, n_rg
        self.n = n_az * n_rg

    def close(self) -> None:
        if self.handle:
            lib.csar_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def csar_plan_create(geometry, flags: int = 0) -> Plan:
    p = params_of(geometry)
    h = ctypes.c_void_p()
    _check(lib.csar_plan_create(ctypes.byref(p), flags, ctypes.byref(h)), "csar_plan_create")
    return Plan(h.value, p.n_az, p.n_rg)


def csar_plan_destroy(plan: Plan) -> None:
    plan.close()


def _opts(K, iters, mu_mode, mu, thresh) -> Opts:
    return Opts(int(K), int(iters), MU_MODES[mu_mode] if isinstance(mu_mode, str) else int(mu_mode),
                float(mu), THRESH[thresh] if isinstance(thresh, str) else int(thresh))


def csar_G(plan: Plan, x, y=None, stream=None):
    """y = G(x) on [n_az, n_rg] complex64 CUDA tensors (y may be x)."""
    import torch
    _need(x, torch.complex64, plan.n, "x")
    y = torch.empty_like(x) if y is None else y
    _need(y, torch.complex64, plan.n, "y")
    _check(lib.csar_G(plan.handle, _ptr(x), _ptr(y), _stream(stream)), "csar_G")
    return y


def csar_G_noalloc(geometry, x, y=None, stream=None):
    """y = G(x) without a plan and without any device allocation by the library
    (tables in a static device array; calls must not overlap on the GPU)."""
    import torch
    p = params_of(geometry)
    n = p.n_az * p.n_rg
    _need(x, torch.complex64, n, "x")
    y = torch.empty_like(x) if y is None else y
    _need(y, torch.complex64, n, "y")
    _check(lib.csar_G_noalloc(ctypes.byref(p), _ptr(x), _ptr(y), _stream(stream)), "csar_G_noalloc")
    return y


def csar_echo_points(geometry, rows, cols, amps, out=None, accumulate: bool = False, stream=None):
    """Raw echo [n_az, n_rg] complex64 (CUDA tensor) of point targets on image pixels
    (rows, cols; complex amplitudes amps) from the exact stripmap model; written into
    ``out`` (or added to it with accumulate=True)."""
    import torch
    p = params_of(geometry)
    rows = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1)
    cols = np.ascontiguousarray(cols, dtype=np.int32).reshape(-1)
    a = np.ascontiguousarray(np.asarray(amps, dtype=np.complex64).reshape(-1)).view(np.float32)
    if not (rows.size == cols.size == a.size // 2):
        raise ValueError("rows, cols and amps must have the same length")
    if out is None:
        out = torch.empty((p.n_az, p.n_rg), dtype=torch.complex64, device="cuda")
    _need(out, torch.complex64, p.n_az * p.n_rg, "out")
    _check(lib.csar_echo_points(ctypes.byref(p), rows.ctypes.data, cols.ctypes.data, a.ctypes.data,
                                rows.size, _ptr(out), int(bool(accumulate)), _stream(stream)),
           "csar_echo_points")
    return out


def csar_M(plan: Plan, y, x=None, stream=None):
    """x = M(y) = G^H(y) on [n_az, n_rg] complex64 CUDA tensors (x may be y)."""
    import torch
    _need(y, torch.complex64, plan.n, "y")
    x = torch.empty_like(y) if x is None else x
    _need(x, torch.complex64, plan.n, "x")
    _check(lib.csar_M(plan.handle, _ptr(y), _ptr(x), _stream(stream)), "csar_M")
    return x


def csar_ita_step(plan: Plan, Y, mask_bits, X, K: int, mu_mode="fixed", mu: float = 1.0,
                  thresh="soft", sigma=None, stream=None):
    """One ITA iteration in place on X (complex64 CUDA); mask_bits: int32 CUDA tensor
    of n/32 packed words.  sigma: optional float32 CUDA tensor of 1 element."""
    import torch
    _need(Y, torch.complex64, plan.n, "Y")
    _need(X, torch.complex64, plan.n, "X")
    _need(mask_bits, torch.int32, plan.n // 32, "mask_bits")
    o = _opts(K, 1, mu_mode, mu, thresh)
    sp = ctypes.c_void_p(None) if sigma is None else _ptr(sigma)
    _check(lib.csar_ita_step(plan.handle, _ptr(Y), _ptr(mask_bits), _ptr(X), ctypes.byref(o), sp,
                             _stream(stream)), "csar_ita_step")
    return X


def _stats_struct(iters: int):
    arrs = {"resid_sq": np.zeros(iters, np.float64), "mu": np.zeros(iters, np.float32),
            "sigma": np.zeros(iters, np.float32), "nnz": np.zeros(iters, np.int64)}
    st = Stats(arrs["resid_sq"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
               arrs["mu"].ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
               arrs["sigma"].ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
               arrs["nnz"].ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return st, arrs


def csar_solve(plan: Plan, Y, mask_bits, K: int, iters: int, mu_mode="fixed", mu: float = 1.0,
               thresh="soft", X=None, stats: bool = False, stream=None):
    """Algorithm 1 from X = 0 for `iters` iterations; returns X (and the per-iteration
    statistics dict when stats=True, which synchronises the stream)."""
    import torch
    _need(Y, torch.complex64, plan.n, "Y")
    _need(mask_bits, torch.int32, plan.n // 32, "mask_bits")
    X = torch.empty_like(Y) if X is None else X
    _need(X, torch.complex64, plan.n, "X")
    o = _opts(K, iters, mu_mode, mu, thresh)
    st, arrs = _stats_struct(max(iters, 1)) if stats else (None, None)
    _check(lib.csar_solve(plan.handle, _ptr(Y), _ptr(mask_bits), _ptr(X), ctypes.byref(o),
                          ctypes.byref(st) if st is not None else None, _stream(stream)),
           "csar_solve")
    return (X, arrs) if stats else X


def csar_solve_host(plan: Plan, Y: np.ndarray, mask_bits: np.ndarray, K: int, iters: int,
                    mu_mode="fixed", mu: float = 1.0, thresh="soft", X: np.ndarray | None = None,
                    stats: bool = False, stream=None):
    """csar_solve from host numpy buffers (complex64 Y, uint32 mask words); returns X."""
    Y = np.ascontiguousarray(Y, dtype=np.complex64)
    mask_bits = np.ascontiguousarray(mask_bits, dtype=np.uint32)
    if Y.size != plan.n or mask_bits.size != plan.n // 32:
        raise ValueError("Y / mask_bits size does not match the plan")
    if X is None:
        X = np.empty(plan.n, dtype=np.complex64)
    o = _opts(K, iters, mu_mode, mu, thresh)
    st, arrs = _stats_struct(max(iters, 1)) if stats else (None, None)
    _check(lib.csar_solve_host(plan.handle, ctypes.c_void_p(Y.ctypes.data),
                               ctypes.c_void_p(mask_bits.ctypes.data), ctypes.c_void_p(X.ctypes.data),
                               ctypes.byref(o), ctypes.byref(st) if st is not None else None,
                               _stream(stream)), "csar_solve_host")
    return (X, arrs) if stats else X


def csar_solve_profile(plan: Plan, Y, mask_bits, K: int, iters: int, mu_mode="fixed",
                       mu: float = 1.0, thresh="soft", X=None, stream=None):
    """csar_solve with CUDA events around every pass; returns (X, {pass: ms summed})."""
    import torch
    X = torch.empty_like(Y) if X is None else X
    o = _opts(K, iters, mu_mode, mu, thresh)
    ms = (ctypes.c_float * N_PASSES)()
    _check(lib.csar_solve_profile(plan.handle, _ptr(Y), _ptr(mask_bits), _ptr(X), ctypes.byref(o),
                                  ms, N_PASSES, _stream(stream)), "csar_solve_profile")
    return X, dict(zip(PASS_NAMES, [float(v) for v in ms]))


def csar_plan_check(plan: Plan) -> None:
    _check(lib.csar_plan_check(plan.handle), "csar_plan_check")


def csar_plan_set_pulse(plan: Plan, spectrum=None) -> None:
    """Range spectrum of a recorded (non-chirp) transmitted pulse for a range-Doppler
    plan, n_rg complex values in FFT bin order (None: back to the chirp filter)."""
    if spectrum is None:
        _check(lib.csar_plan_set_pulse(plan.handle, None), "csar_plan_set_pulse")
        return
    s = np.ascontiguousarray(np.asarray(spectrum).astype(np.complex64).reshape(-1))
    if s.size != plan.n_rg:
        raise ValueError(f"pulse spectrum needs {plan.n_rg} bins, got {s.size}")
    _check(lib.csar_plan_set_pulse(plan.handle, ctypes.c_void_p(s.ctypes.data)), "csar_plan_set_pulse")


def csar_debug_fail_alloc(n: int) -> None:
    """Make the n-th device allocation of the library from now on fail as out of memory
    (0: off)."""
    _check(lib.csar_debug_fail_alloc(int(n)), "csar_debug_fail_alloc")


def csar_debug_selection_enable(plan: Plan, capacity: int) -> None:
    """Record the union the selection ranks in every later ITA iteration of the plan
    (capacity entries; 0 turns the record off)."""
    _check(lib.csar_debug_selection_enable(plan.handle, int(capacity)), "csar_debug_selection_enable")


def csar_debug_selection_read(plan: Plan, capacity: int) -> dict:
    """The last recorded union: flat indices, b (complex64) and keys (uint32) as the
    selection kernels formed them, plus sigma2_key, mu and sigma of that iteration."""
    idx = np.zeros(capacity, dtype=np.uint32)
    b = np.zeros(capacity, dtype=np.complex64)
    key = np.zeros(capacity, dtype=np.uint32)
    cnt, s2 = ctypes.c_int64(0), ctypes.c_uint32(0)
    mu, sig = ctypes.c_float(0), ctypes.c_float(0)
    _check(lib.csar_debug_selection_read(plan.handle, idx.ctypes.data, b.ctypes.data, key.ctypes.data,
                                         int(capacity), ctypes.byref(cnt), ctypes.byref(s2),
                                         ctypes.byref(mu), ctypes.byref(sig)),
           "csar_debug_selection_read")
    m = min(int(cnt.value), capacity)
    return {"idx": idx[:m], "b": b[:m], "key": key[:m], "count": int(cnt.value),
            "sigma2_key": int(s2.value), "mu": float(mu.value), "sigma": float(sig.value)}


def csar_version() -> int:
    return int(lib.csar_version())


def pack_mask_torch(mask_bool):
    """Pack a boolean [n_az, n_rg] torch mask into int32 words (bit j of word w is
    element 32 w + j) on the mask's device."""
    import torch
    flat = mask_bool.reshape(-1, 32).to(torch.int64)
    weights = (torch.ones(32, dtype=torch.int64, device=flat.device) << torch.arange(
        32, device=flat.device))
    words = (flat * weights).sum(dim=1)
    words = torch.where(words >= 2 ** 31, words - 2 ** 32, words)
    return words.to(torch.int32)


# ----------------------------------------------------------------------------- autofocus

def csar_af_solve(plan: Plan, Y, mask_bits, theta, K: int, iters: int, mu: float = 1.0,
                  checkpoint: bool = True, X=None, stream=None):
    """X^(I) of the ITA for the observation S . (exp(j theta) G X) (soft threshold,
    fixed step); keeps per-iteration checkpoints in the plan for csar_af_backward."""
    import torch
    _need(Y, torch.complex64, plan.n, "Y")
    _need(mask_bits, torch.int32, plan.n // 32, "mask_bits")
    _need(theta, torch.float32, plan.n_az, "theta")
    X = torch.empty_like(Y) if X is None else X
    o = _opts(K, iters, "fixed", mu, "soft")
    _check(lib.csar_af_solve(plan.handle, _ptr(Y), _ptr(mask_bits), _ptr(theta), _ptr(X),
                             ctypes.byref(o), int(bool(checkpoint)), _stream(stream)), "csar_af_solve")
    return X


def csar_af_loss(plan: Plan, Y, mask_bits, theta, X, grads: bool = True, stream=None):
    """(loss, grad_X, grad_theta) of ||S.(exp(-j theta) Y - G X)||^2 (device tensors)."""
    import torch
    _need(X, torch.complex64, plan.n, "X")
    loss = torch.zeros(1, dtype=torch.float64, device=X.device)
    gx = torch.empty_like(X) if grads else None
    gt = torch.empty(plan.n_az, dtype=torch.float32, device=X.device) if grads else None
    _check(lib.csar_af_loss(plan.handle, _ptr(Y), _ptr(mask_bits), _ptr(theta), _ptr(X), _ptr(loss),
                            _ptr(gx) if grads else None, _ptr(gt) if grads else None,
                            _stream(stream)), "csar_af_loss")
    return loss, gx, gt


def csar_af_backward(plan: Plan, Y, mask_bits, theta, Xbar, theta_bar=None, X0bar=None, stream=None):
    """Adjoint of the last checkpointed csar_af_solve: adds into theta_bar (returned)."""
    import torch
    _need(Xbar, torch.complex64, plan.n, "Xbar")
    theta_bar = (torch.zeros(plan.n_az, dtype=torch.float32, device=Xbar.device)
                 if theta_bar is None else theta_bar)
    _check(lib.csar_af_backward(plan.handle, _ptr(Y), _ptr(mask_bits), _ptr(theta), _ptr(Xbar),
                                _ptr(theta_bar), _ptr(X0bar) if X0bar is not None else None,
                                _stream(stream)), "csar_af_backward")
    return theta_bar


def _autograd():
    import torch

    class ITAUnroll(torch.autograd.Function):
        """X^(I)(theta) of the unrolled ITA; backward through the checkpoints."""

        @staticmethod
        def forward(ctx, theta, plan, Y, mask_bits, K, iters, mu):
            X = csar_af_solve(plan, Y, mask_bits, theta.detach(), K, iters, mu, checkpoint=True)
            ctx.plan, ctx.Y, ctx.mask = plan, Y, mask_bits
            ctx.save_for_backward(theta)
            return X

        @staticmethod
        def backward(ctx, gX):
            (theta,) = ctx.saved_tensors
            tb = csar_af_backward(ctx.plan, ctx.Y, ctx.mask, theta.detach(), gX.contiguous())
            return tb, None, None, None, None, None, None

    class AutofocusLoss(torch.autograd.Function):
        """||S.(exp(-j theta) Y - G X)||^2 with its analytic gradients."""

        @staticmethod
        def forward(ctx, X, theta, plan, Y, mask_bits):
            loss, gx, gt = csar_af_loss(plan, Y, mask_bits, theta.detach(), X.detach())
            ctx.save_for_backward(gx, gt)
            return loss.reshape(())

        @staticmethod
        def backward(ctx, gl):
            gx, gt = ctx.saved_tensors
            return gl.to(gx.real.dtype) * gx, gl.to(gt.dtype) * gt, None, None, None

    return ITAUnroll, AutofocusLoss


def autofocus_loss(plan: Plan, Y, mask_bits, theta, K: int, iters: int, mu: float = 1.0):
    """L(theta) = ||S.(exp(-j theta) Y - G X_I(theta))||^2 through the unrolled ITA,
    differentiable with respect to theta (torch.autograd)."""
    ITAUnroll, AutofocusLoss = _autograd()
    X = ITAUnroll.apply(theta, plan, Y, mask_bits, K, iters, mu)
    return AutofocusLoss.apply(X, theta, plan, Y, mask_bits)


# ----------------------------------------------------------------------------- batches

class Batch:
    """Owns a csar_batch handle (one plan per patch)."""

    def __init__(self, handle: int, shapes):
        self.handle = ctypes.c_void_p(handle)
        self.shapes = list(shapes)

    def close(self) -> None:
        if self.handle:
            lib.csar_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def csar_batch_create(geometries, flags: int = 0) -> Batch:
    arr = (Params * len(geometries))(*[params_of(g) for g in geometries])
    h = ctypes.c_void_p()
    _check(lib.csar_batch_create(arr, len(geometries), flags, ctypes.byref(h)), "csar_batch_create")
    return Batch(h.value, [(g.n_az, g.n_rg) for g in geometries])


def csar_solve_batched(batch: Batch, Ys, masks, Ks, iters: int, mu_mode="fixed", mu: float = 1.0,
                       thresh="soft", Xs=None, stream=None):
    """Algorithm 1 on every patch together (one graph launch per iteration)."""
    import torch
    n = len(batch.shapes)
    Xs = [torch.empty_like(y) for y in Ys] if Xs is None else Xs
    for i, (na, nr) in enumerate(batch.shapes):
        _need(Ys[i], torch.complex64, na * nr, f"Y[{i}]")
        _need(masks[i], torch.int32, na * nr // 32, f"mask[{i}]")
        _need(Xs[i], torch.complex64, na * nr, f"X[{i}]")
    vpa = ctypes.c_void_p * n
    ys = vpa(*[y.data_ptr() for y in Ys])
    ms = vpa(*[m.data_ptr() for m in masks])
    xs = vpa(*[x.data_ptr() for x in Xs])
    ks = (ctypes.c_int64 * n)(*[int(k) for k in Ks])
    o = _opts(0, iters, mu_mode, mu, thresh)
    _check(lib.csar_solve_batched(batch.handle, ys, ms, xs, ks, ctypes.byref(o), _stream(stream)),
           "csar_solve_batched")
    return Xs


def csar_batch_check(batch: Batch) -> None:
    _check(lib.csar_batch_check(batch.handle), "csar_batch_check")


def csar_selftest_wait_timeout(limit_ms: int = 20) -> int:
    """Run the column-pass exchange wait on an mbarrier nothing arrives at; returns the
    status (CSAR_E_TIMEOUT = 5 is the expected outcome)."""
    return int(lib.csar_selftest_wait_timeout(int(limit_ms)))


def csar_autotune(geometry, iters: int = 10) -> int:
    """Time every column-pass configuration for this shape; later plans use the fastest.
    Returns the cluster size of the chosen configuration."""
    p = params_of(geometry)
    out = ctypes.c_int32(0)
    _check(lib.csar_autotune(ctypes.byref(p), int(iters), ctypes.byref(out)), "csar_autotune")
    return int(out.value)


def plan_col_cluster(p: int) -> int:
    """csar_plan_create flag forcing the column-pass cluster size."""
    return int(p) << 8


# csar_plan_create flag: column-pass CTAs of 4096 complex values (half-width tiles)
PLAN_COL_HALF_TILE = 1 << 16
# csar_plan_create flag: column-pass CTAs of 16384 complex values (double-width tiles)
PLAN_COL_WIDE_TILE = 1 << 18
# csar_plan_create flag: G / M are the range-Doppler operator pair with sinc RCMC
PLAN_RDA = 1 << 17
# csar_plan_create flags: persistent, tensor-copy-fed column passes, or never
PLAN_COL_PERSIST = 1 << 19
PLAN_COL_NO_PERSIST = 1 << 20
# csar_plan_create flag: the configuration of a member of a one-launch-per-pass batch
# (bit-identical to what csar_solve_batched computes for that patch)
PLAN_BATCH_MEMBER = 1 << 21
