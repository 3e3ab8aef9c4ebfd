"""ctypes binding of libsslbm.so (include/sslbm.h), with the C entry points' names.

Argument marshalling only: every computation runs in the library's CUDA kernels.
PyTorch supplies device memory (the workspace) and streams.  If the library has not
been built, the first call raises; there is no CPU fallback.

Functions mirror the C ABI one to one (``sslbm_create``, ``sslbm_step``,
``bgk_step``, ``sslbm_read`` ...) and raise ``SslbmError`` on a negative status.
``Solver`` bundles a handle with its torch-allocated workspace for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# SSLBM_LIBRARY selects another build of the same library (the index-checked debug build)
LIB_PATH = os.environ.get("SSLBM_LIBRARY") or os.path.join(_PKG, "libsslbm.so")

# constants of include/sslbm.h
SSLBM_OK = 0
(SSLBM_ERR_BAD_ARG, SSLBM_ERR_UNSTABLE, SSLBM_ERR_CUDA, SSLBM_ERR_TIMEOUT, SSLBM_ERR_NONFINITE,
 SSLBM_ERR_WORKSPACE, SSLBM_ERR_UNSUPPORTED, SSLBM_ERR_STATE) = (-1, -2, -3, -4, -5, -6, -7, -8)
BC_PERIODIC, BC_NOFLUX = 0, 1
FP64, FP32, FP32_DEV, FP32_KAHAN, FP32_SPLIT, FP64_DW = 0, 1, 2, 3, 4, 5
SCHEME_SSLBM, SCHEME_BGK = 0, 1
S, E, I, R, D, NCOMP = 0, 1, 2, 3, 4, 5
ALL = -1
DT_F64, DT_F32 = 0, 1
WANT_SSLBM, WANT_BGK = 1, 2
LATTICE_D2Q5, LATTICE_D2Q9, LATTICE_D2Q5_SLBM, LATTICE_D2Q5_VARD = 0, 1, 2, 3
MAX_DEPTH = 8
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp32_dev": FP32_DEV, "fp32_kahan": FP32_KAHAN, "fp32_split": FP32_SPLIT,
              "fp64_dw": FP64_DW}

# every symbol include/sslbm.h declares
EXPORTS = ("sslbm_strerror", "sslbm_last_error", "sslbm_version", "sslbm_workspace_bytes",
           "sslbm_create", "sslbm_set_stream", "sslbm_destroy", "sslbm_write", "sslbm_read",
           "sslbm_set_diffusivity_scale", "sslbm_step", "bgk_step", "sslbm_steps_done",
           "sslbm_checkpoint_bytes", "sslbm_checkpoint_save", "sslbm_checkpoint_load",
           "sslbm_debug_bounds", "sslbm_debug_bounds_probe",
           "sslbm_diagnostics", "sslbm_set_fused_diagnostics",
           "sslbm_get_fused_diagnostics", "sslbm_set_blocking",
           "sslbm_get_blocking", "sslbm_diagnostics_noalloc", "sslbm_autotune",
           "sslbm_ensemble_workspace_bytes", "sslbm_ensemble_create", "sslbm_ensemble_destroy",
           "sslbm_ensemble_set_tiling", "sslbm_ensemble_get_tiling",
           "sslbm_ensemble_set_wait_limit", "sslbm_ensemble_write", "sslbm_ensemble_read",
           "sslbm_ensemble_run", "sslbm_ensemble_diagnostics", "sslbm_ensemble_autotune",
           "sslbm_ensemble_steps_done", "sslbm_ensemble_checkpoint_bytes", "sslbm_ensemble_checkpoint_save",
           "sslbm_ensemble_checkpoint_load", "sslbm_fno_workspace_bytes", "sslbm_fno_create",
           "sslbm_fno_destroy", "sslbm_fno_num_params", "sslbm_fno_set_params",
           "sslbm_fno_get_params", "sslbm_fno_get_grads", "sslbm_fno_make_input",
           "sslbm_fno_forward", "sslbm_fno_backward", "sslbm_fno_set_adam", "sslbm_fno_set_loss_weights",
           "sslbm_fno_set_wait_limit",
           "sslbm_fno_infer", "sslbm_fno_fused",
           "sslbm_fno_train_step", "sslbm_fno_check_project", "sslbm_surrogate_rollout",
           "sslbm_fd4_workspace_bytes", "sslbm_fd4_create", "sslbm_fd4_destroy", "sslbm_fd4_write",
           "sslbm_fd4_read", "sslbm_fd4_step", "sslbm_fd4_steps_done", "sslbm_fd4_set_order")


class RolloutStats(ctypes.Structure):
    _fields_ = [("surrogate_steps", ctypes.c_int64), ("fallbacks", ctypes.c_int64),
                ("failed_conservation", ctypes.c_int64), ("failed_nonnegativity", ctypes.c_int64),
                ("max_mass_residual", ctypes.c_double), ("max_neg_residual", ctypes.c_double)]


class SslbmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {sslbm_strerror(status)} ({status}): {detail}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("dx", ctypes.c_double),
                ("dt", ctypes.c_double), ("bc", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("schemes", ctypes.c_int32), ("lattice", ctypes.c_int32)]


class Scenario(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("dx", ctypes.c_double),
                ("dt", ctypes.c_double), ("beta", ctypes.c_double), ("alpha", ctypes.c_double),
                ("gamma", ctypes.c_double), ("phi", ctypes.c_double), ("d", ctypes.c_double * 5),
                ("s_ref", ctypes.c_double)]


class FnoConfig(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("width", ctypes.c_int32), ("modes", ctypes.c_int32),
                ("layers", ctypes.c_int32), ("hidden", ctypes.c_int32), ("max_batch", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("alpha", ctypes.c_double), ("gamma", ctypes.c_double),
                ("phi", ctypes.c_double), ("d", ctypes.c_double * 5), ("tau", ctypes.c_double * 4),
                ("s_ref", ctypes.c_double), ("use_tau", ctypes.c_int32), ("strict", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p


def load(path: str = LIB_PATH):
    """Load libsslbm.so (raises if it is missing: build it with paper_2603_19789_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -m paper_2603_19789_gb300.build` (no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        i32, i64 = ctypes.c_int, ctypes.c_int64
        sig = {
            "sslbm_strerror": (ctypes.c_char_p, [i32]),
            "sslbm_last_error": (ctypes.c_char_p, []),
            "sslbm_version": (i32, []),
            "sslbm_workspace_bytes": (i32, [ctypes.POINTER(Grid), ctypes.POINTER(ctypes.c_size_t)]),
            "sslbm_create": (i32, [ctypes.POINTER(Grid), ctypes.POINTER(Params), _vp, ctypes.c_size_t,
                                   _vp, ctypes.POINTER(_vp)]),
            "sslbm_set_stream": (i32, [_vp, _vp]),
            "sslbm_destroy": (None, [_vp]),
            "sslbm_write": (i32, [_vp, i32, i32, _vp, i32, i32]),
            "sslbm_read": (i32, [_vp, i32, i32, _vp, i32, i32]),
            "sslbm_set_diffusivity_scale": (i32, [_vp, _vp, _vp, i32, i32]),
            "sslbm_step": (i32, [_vp, i64]),
            "bgk_step": (i32, [_vp, i64]),
            "sslbm_steps_done": (i64, [_vp, i32]),
            "sslbm_debug_bounds": (i32, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i32)]),
            "sslbm_debug_bounds_probe": (i32, [ctypes.c_longlong, ctypes.c_longlong]),
            "sslbm_checkpoint_bytes": (i32, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
            "sslbm_checkpoint_save": (i32, [_vp, _vp, ctypes.c_size_t, i32]),
            "sslbm_checkpoint_load": (i32, [_vp, _vp, ctypes.c_size_t, i32]),
            "sslbm_diagnostics": (i32, [_vp, i32, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
            "sslbm_set_fused_diagnostics": (i32, [_vp, i32]),
            "sslbm_get_fused_diagnostics": (i32, [_vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "sslbm_set_blocking": (i32, [_vp, i32, i32]),
            "sslbm_get_blocking": (i32, [_vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "sslbm_autotune": (i32, [_vp, ctypes.c_double, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(ctypes.c_double)]),
            "sslbm_ensemble_workspace_bytes": (i32, [i32, _vp, i32, ctypes.POINTER(ctypes.c_size_t)]),
            "sslbm_fd4_workspace_bytes": (i32, [ctypes.POINTER(Grid), ctypes.POINTER(ctypes.c_size_t)]),
            "sslbm_fd4_create": (i32, [ctypes.POINTER(Grid), ctypes.POINTER(Params), _vp, ctypes.c_size_t, _vp,
                                       ctypes.POINTER(_vp)]),
            "sslbm_fd4_destroy": (None, [_vp]),
            "sslbm_fd4_write": (i32, [_vp, _vp, i32, i32]),
            "sslbm_fd4_read": (i32, [_vp, _vp, i32, i32]),
            "sslbm_fd4_step": (i32, [_vp, ctypes.c_int64]),
            "sslbm_fd4_steps_done": (ctypes.c_int64, [_vp]),
            "sslbm_fd4_set_order": (i32, [_vp, i32]),
            "sslbm_ensemble_create": (i32, [i32, _vp, i32, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
            "sslbm_ensemble_destroy": (None, [_vp]),
            "sslbm_ensemble_set_tiling": (i32, [_vp, i32, i32]),
            "sslbm_ensemble_get_tiling": (i32, [_vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "sslbm_ensemble_set_wait_limit": (i32, [_vp, ctypes.c_longlong, ctypes.c_longlong]),
            "sslbm_ensemble_write": (i32, [_vp, i32, _vp, i32, i32]),
            "sslbm_ensemble_read": (i32, [_vp, i32, _vp, i32, i32]),
            "sslbm_ensemble_run": (i32, [_vp, i64]),
            "sslbm_ensemble_diagnostics": (i32, [_vp, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_double)]),
            "sslbm_ensemble_autotune": (i32, [_vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                              ctypes.POINTER(ctypes.c_double)]),
            "sslbm_ensemble_steps_done": (i64, [_vp]),
            "sslbm_ensemble_checkpoint_bytes": (i32, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
            "sslbm_ensemble_checkpoint_save": (i32, [_vp, _vp, ctypes.c_size_t, i32]),
            "sslbm_ensemble_checkpoint_load": (i32, [_vp, _vp, ctypes.c_size_t, i32]),
            "sslbm_fno_workspace_bytes": (i32, [ctypes.POINTER(FnoConfig), ctypes.POINTER(ctypes.c_size_t)]),
            "sslbm_fno_create": (i32, [ctypes.POINTER(FnoConfig), _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
            "sslbm_fno_destroy": (None, [_vp]),
            "sslbm_fno_num_params": (i64, [_vp]),
            "sslbm_fno_set_params": (i32, [_vp, _vp, i32]),
            "sslbm_fno_get_params": (i32, [_vp, _vp, i32]),
            "sslbm_fno_get_grads": (i32, [_vp, _vp, i32]),
            "sslbm_fno_make_input": (i32, [_vp, i32, _vp, _vp, _vp, _vp]),
            "sslbm_fno_forward": (i32, [_vp, i32, _vp, _vp]),
            "sslbm_fno_backward": (i32, [_vp, i32, _vp, _vp]),
            "sslbm_fno_set_adam": (i32, [_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
            "sslbm_fno_set_loss_weights": (i32, [_vp, ctypes.c_float, ctypes.c_float]),
            "sslbm_fno_set_wait_limit": (i32, [_vp, ctypes.c_longlong, i32]),
            "sslbm_fno_infer": (i32, [_vp, i32, _vp, _vp]),
            "sslbm_fno_fused": (i32, [_vp]),
            "sslbm_fno_train_step": (i32, [_vp, i32, _vp, _vp, _vp, _vp, ctypes.c_float,
                                           ctypes.POINTER(ctypes.c_double)]),
            "sslbm_fno_check_project": (i32, [_vp, i32, _vp, _vp, i32, ctypes.POINTER(ctypes.c_double)]),
            "sslbm_surrogate_rollout": (i32, [_vp, _vp, i32, i32, i32, _vp, _vp, _vp, _vp, _vp, ctypes.c_double,
                                              ctypes.c_double, i32, _vp, _vp, ctypes.POINTER(RolloutStats)]),
            "sslbm_diagnostics_noalloc": (i32, [_vp, i32, i64, i64, ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_double), _vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != SSLBM_OK:
        raise SslbmError(status, where, sslbm_last_error())


def sslbm_strerror(status: int) -> str:
    return load().sslbm_strerror(int(status)).decode()


def sslbm_last_error() -> str:
    return load().sslbm_last_error().decode()


def sslbm_version() -> int:
    return int(load().sslbm_version())


def make_grid(nx, ny, dx=1.0, dt=1.0, bc=BC_PERIODIC, precision=FP64, schemes=WANT_SSLBM,
              lattice=LATTICE_D2Q5) -> Grid:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    return Grid(int(nx), int(ny), float(dx), float(dt), int(bc), int(precision), int(schemes), int(lattice))


def make_params(beta, alpha, gamma, phi, d=None, tau=None, s_ref=1.0, strict=False) -> Params:
    p = Params()
    p.beta, p.alpha, p.gamma, p.phi = float(beta), float(alpha), float(gamma), float(phi)
    if tau is not None:
        p.use_tau = 1
        for c in range(4):
            p.tau[c] = float(tau[c])
    else:
        dd = list(d) + [0.0] * (5 - len(d))
        for c in range(5):
            p.d[c] = float(dd[c])
    p.s_ref = float(s_ref)
    p.strict = 1 if strict else 0
    return p


def sslbm_workspace_bytes(grid: Grid) -> int:
    n = ctypes.c_size_t(0)
    _check(load().sslbm_workspace_bytes(ctypes.byref(grid), ctypes.byref(n)), "sslbm_workspace_bytes")
    return int(n.value)


def sslbm_create(grid: Grid, params: Params, ws_ptr: int, ws_bytes: int, stream: int = 0):
    h = _vp()
    _check(load().sslbm_create(ctypes.byref(grid), ctypes.byref(params), _vp(ws_ptr), int(ws_bytes),
                               _vp(stream), ctypes.byref(h)), "sslbm_create")
    return h


def sslbm_set_stream(h, stream: int):
    _check(load().sslbm_set_stream(h, _vp(stream)), "sslbm_set_stream")


def sslbm_destroy(h):
    if h:
        load().sslbm_destroy(h)


def _buffer(a):
    """(pointer, on_device, dtype code, nbytes) of a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        code = {np.dtype(np.float64): DT_F64, np.dtype(np.float32): DT_F32}.get(a.dtype)
        if code is None:
            raise TypeError(f"unsupported dtype {a.dtype}")
        return a.ctypes.data, 0, code, a.nbytes
    import torch
    if not isinstance(a, torch.Tensor):
        raise TypeError(type(a))
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    code = {torch.float64: DT_F64, torch.float32: DT_F32}.get(a.dtype)
    if code is None:
        raise TypeError(f"unsupported dtype {a.dtype}")
    return a.data_ptr(), 1 if a.is_cuda else 0, code, a.numel() * a.element_size()


def sslbm_write(h, scheme: int, comp: int, src):
    ptr, dev, code, _ = _buffer(src)
    _check(load().sslbm_write(h, int(scheme), int(comp), _vp(ptr), code, dev), "sslbm_write")


def sslbm_read(h, scheme: int, comp: int, dst):
    ptr, dev, code, _ = _buffer(dst)
    _check(load().sslbm_read(h, int(scheme), int(comp), _vp(ptr), code, dev), "sslbm_read")
    return dst


def sslbm_set_diffusivity_scale(h, kx, ky=None):
    """Per-cell diffusivity scale fields (ny, nx) of a LATTICE_D2Q5_VARD solver; ky=None uses
    kx on both axes.  numpy arrays or torch tensors (host or device) of one dtype."""
    px, dx, cx, nx_bytes = _buffer(kx)
    py, cy_code = 0, cx
    if ky is not None:
        py, dy, cy_code, ny_bytes = _buffer(ky)
        if dy != dx or cy_code != cx or ny_bytes != nx_bytes:
            raise ValueError("kx and ky must share dtype, size and location")
    _check(load().sslbm_set_diffusivity_scale(h, _vp(px), _vp(py) if ky is not None else None, cx, dx),
           "sslbm_set_diffusivity_scale")


def sslbm_step(h, n: int):
    _check(load().sslbm_step(h, int(n)), "sslbm_step")


def bgk_step(h, n: int):
    _check(load().bgk_step(h, int(n)), "bgk_step")


def sslbm_steps_done(h, scheme: int = SCHEME_SSLBM) -> int:
    return int(load().sslbm_steps_done(h, int(scheme)))


def _raw(a):
    """(pointer, on_device, nbytes) of a contiguous numpy array or torch tensor of any dtype."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0, a.nbytes
    import torch
    if not isinstance(a, torch.Tensor):
        raise TypeError(type(a))
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr(), 1 if a.is_cuda else 0, a.numel() * a.element_size()


def sslbm_debug_bounds():
    """Index checks of the debug build since the last call: {count, value, limit, site}
    (SslbmError with SSLBM_ERR_UNSUPPORTED from a release build)."""
    c, v, lim = ctypes.c_longlong(0), ctypes.c_longlong(0), ctypes.c_longlong(0)
    site = ctypes.c_int(0)
    _check(load().sslbm_debug_bounds(ctypes.byref(c), ctypes.byref(v), ctypes.byref(lim), ctypes.byref(site)),
           "sslbm_debug_bounds")
    return {"count": int(c.value), "value": int(v.value), "limit": int(lim.value), "site": int(site.value)}


def sslbm_debug_bounds_probe(value: int, limit: int):
    _check(load().sslbm_debug_bounds_probe(int(value), int(limit)), "sslbm_debug_bounds_probe")


def sslbm_checkpoint_bytes(h) -> int:
    n = ctypes.c_size_t(0)
    _check(load().sslbm_checkpoint_bytes(h, ctypes.byref(n)), "sslbm_checkpoint_bytes")
    return int(n.value)


def sslbm_checkpoint_save(h, dst):
    """State and step counters into dst (a uint8 numpy array or torch tensor, host or device)."""
    ptr, dev, nbytes = _raw(dst)
    _check(load().sslbm_checkpoint_save(h, _vp(ptr), nbytes, dev), "sslbm_checkpoint_save")
    return dst


def sslbm_checkpoint_load(h, src):
    ptr, dev, nbytes = _raw(src)
    _check(load().sslbm_checkpoint_load(h, _vp(ptr), nbytes, dev), "sslbm_checkpoint_load")


def sslbm_diagnostics(h, scheme: int = SCHEME_SSLBM):
    tot = (ctypes.c_double * 5)()
    pk = ctypes.c_double(0.0)
    _check(load().sslbm_diagnostics(h, int(scheme), tot, ctypes.byref(pk)), "sslbm_diagnostics")
    return np.array(tot[:]), float(pk.value)


def sslbm_diagnostics_noalloc(fields, stream: int = 0):
    """Totals and peak infected of a device tensor of shape (5, ny, nx) (float64 or
    float32) through the allocation-free entry point; returns (totals, peak_I)."""
    ptr, dev, code, _ = _buffer(fields)
    if not dev:
        raise ValueError("fields must be a device tensor")
    if fields.dim() != 3 or fields.shape[0] != 5:
        raise ValueError("fields must have shape (5, ny, nx)")
    tot = (ctypes.c_double * 5)()
    pk = ctypes.c_double(0.0)
    _check(load().sslbm_diagnostics_noalloc(_vp(ptr), code, int(fields.shape[2]), int(fields.shape[1]),
                                            tot, ctypes.byref(pk), _vp(stream)),
           "sslbm_diagnostics_noalloc")
    return np.array(tot[:]), float(pk.value)


def sslbm_set_fused_diagnostics(h, on: bool):
    _check(load().sslbm_set_fused_diagnostics(h, 1 if on else 0), "sslbm_set_fused_diagnostics")


def sslbm_get_fused_diagnostics(h):
    """(on, ready): fused diagnostics on, and the current state's diagnostics left by the last pass."""
    on, ready = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().sslbm_get_fused_diagnostics(h, ctypes.byref(on), ctypes.byref(ready)),
           "sslbm_get_fused_diagnostics")
    return bool(on.value), bool(ready.value)


def sslbm_set_blocking(h, k: int, seg_rows: int = 0):
    _check(load().sslbm_set_blocking(h, int(k), int(seg_rows)), "sslbm_set_blocking")


def sslbm_autotune(h, budget_ms: float = 0.0):
    """Time candidate (depth, segment) launches and apply the fastest; returns
    (depth, seg_rows, ms_per_lattice_step)."""
    k, sg, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(load().sslbm_autotune(h, float(budget_ms), ctypes.byref(k), ctypes.byref(sg), ctypes.byref(ms)),
           "sslbm_autotune")
    return int(k.value), int(sg.value), float(ms.value)


def sslbm_get_blocking(h):
    k, s = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().sslbm_get_blocking(h, ctypes.byref(k), ctypes.byref(s)), "sslbm_get_blocking")
    return int(k.value), int(s.value)


class Solver:
    """A handle plus its torch-allocated device workspace.

    rates: (beta, alpha, gamma, phi) in the paper's notation; d: diffusivities of
    S, E, I, R (and D = 0) or tau: relaxation times of S, E, I, R.
    """

    def __init__(self, nx, ny, rates, d=None, tau=None, dx=1.0, dt=1.0, bc=BC_PERIODIC,
                 precision=FP64, schemes=WANT_SSLBM, s_ref=1.0, strict=False, device=None, stream=None,
                 lattice=LATTICE_D2Q5):
        import torch
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        self.grid = make_grid(nx, ny, dx, dt, bc, precision, schemes, lattice)
        self.params = make_params(*rates, d=d, tau=tau, s_ref=s_ref, strict=strict)
        self.nx, self.ny = int(nx), int(ny)
        nbytes = sslbm_workspace_bytes(self.grid)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = sslbm_create(self.grid, self.params, self.ws.data_ptr(), nbytes, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            self.stream.synchronize()
            sslbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def write(self, state, scheme=SCHEME_SSLBM, comp=ALL):
        sslbm_write(self.h, scheme, comp, state)

    def read(self, scheme=SCHEME_SSLBM, comp=ALL, dtype=np.float64):
        shape = (5, self.ny, self.nx) if comp == ALL else (self.ny, self.nx)
        out = np.empty(shape, dtype=dtype)
        return sslbm_read(self.h, scheme, comp, out)

    def set_diffusivity_scale(self, kx, ky=None):
        """Spatially varying (and, with ky, anisotropic) diffusion: d^C k(x) per cell."""
        for f in (kx, ky):
            if f is not None and tuple(f.shape) != (self.ny, self.nx):
                raise ValueError(f"scale field of shape {tuple(f.shape)}, expected {(self.ny, self.nx)}")
        sslbm_set_diffusivity_scale(self.h, kx, ky)

    def step(self, n):
        sslbm_step(self.h, n)

    def bgk_step(self, n):
        bgk_step(self.h, n)

    def diagnostics(self, scheme=SCHEME_SSLBM):
        return sslbm_diagnostics(self.h, scheme)

    def set_fused_diagnostics(self, on=True):
        sslbm_set_fused_diagnostics(self.h, on)

    def get_fused_diagnostics(self):
        return sslbm_get_fused_diagnostics(self.h)

    def set_blocking(self, k, seg_rows=0):
        sslbm_set_blocking(self.h, k, seg_rows)

    def get_blocking(self):
        return sslbm_get_blocking(self.h)

    def autotune(self, budget_ms=0.0):
        return sslbm_autotune(self.h, budget_ms)

    def steps_done(self, scheme=SCHEME_SSLBM):
        return sslbm_steps_done(self.h, scheme)

    def checkpoint(self, on_device=False):
        """The state as stored, with the step counters: a host numpy uint8 array, or a
        device uint8 tensor with on_device=True."""
        n = sslbm_checkpoint_bytes(self.h)
        if on_device:
            buf = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
        else:
            buf = np.empty(n, dtype=np.uint8)
        return sslbm_checkpoint_save(self.h, buf)

    def restore(self, buf):
        """Resume from a checkpoint of a solver with the same grid, precision, lattice,
        boundary and schemes."""
        sslbm_checkpoint_load(self.h, buf)


# ---------------------------------------------------------------------------
# ensembles
# ---------------------------------------------------------------------------

def make_scenarios(specs):
    """specs: iterable of dicts with nx, ny, rates (beta, alpha, gamma, phi), d (4 or 5
    values), optional dx, dt, s_ref."""
    specs = list(specs)
    arr = (Scenario * len(specs))()
    for i, sp in enumerate(specs):
        sc = arr[i]
        sc.nx, sc.ny = int(sp["nx"]), int(sp["ny"])
        sc.dx, sc.dt = float(sp.get("dx", 1.0)), float(sp.get("dt", 1.0))
        sc.beta, sc.alpha, sc.gamma, sc.phi = (float(v) for v in sp["rates"])
        d = list(sp["d"]) + [0.0] * (5 - len(sp["d"]))
        for c in range(5):
            sc.d[c] = float(d[c])
        sc.s_ref = float(sp.get("s_ref", 1.0))
    return arr


def sslbm_ensemble_workspace_bytes(scenarios, precision=FP32) -> int:
    n = ctypes.c_size_t(0)
    _check(load().sslbm_ensemble_workspace_bytes(len(scenarios), ctypes.cast(scenarios, _vp), int(precision),
                                                 ctypes.byref(n)), "sslbm_ensemble_workspace_bytes")
    return int(n.value)


def sslbm_ensemble_create(scenarios, precision, ws_ptr, ws_bytes, stream=0):
    e = _vp()
    _check(load().sslbm_ensemble_create(len(scenarios), ctypes.cast(scenarios, _vp), int(precision), _vp(ws_ptr),
                                        int(ws_bytes), _vp(stream), ctypes.byref(e)), "sslbm_ensemble_create")
    return e


def sslbm_ensemble_destroy(e):
    if e:
        load().sslbm_ensemble_destroy(e)


def sslbm_ensemble_set_tiling(e, depth, seg_rows):
    _check(load().sslbm_ensemble_set_tiling(e, int(depth), int(seg_rows)), "sslbm_ensemble_set_tiling")


def sslbm_ensemble_get_tiling(e):
    d, s = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().sslbm_ensemble_get_tiling(e, ctypes.byref(d), ctypes.byref(s)), "sslbm_ensemble_get_tiling")
    return int(d.value), int(s.value)


def sslbm_ensemble_set_wait_limit(e, spin_limit, stall_item=-1):
    _check(load().sslbm_ensemble_set_wait_limit(e, int(spin_limit), int(stall_item)),
           "sslbm_ensemble_set_wait_limit")


def sslbm_ensemble_write(e, idx, src):
    ptr, dev, code, _ = _buffer(src)
    _check(load().sslbm_ensemble_write(e, int(idx), _vp(ptr), code, dev), "sslbm_ensemble_write")


def sslbm_ensemble_read(e, idx, dst):
    ptr, dev, code, _ = _buffer(dst)
    _check(load().sslbm_ensemble_read(e, int(idx), _vp(ptr), code, dev), "sslbm_ensemble_read")
    return dst


def sslbm_ensemble_run(e, nsteps):
    _check(load().sslbm_ensemble_run(e, int(nsteps)), "sslbm_ensemble_run")


def sslbm_ensemble_diagnostics(e, n):
    tot = (ctypes.c_double * (5 * n))()
    pk = (ctypes.c_double * n)()
    _check(load().sslbm_ensemble_diagnostics(e, tot, pk), "sslbm_ensemble_diagnostics")
    return np.array(tot[:]).reshape(n, 5), np.array(pk[:])


def sslbm_ensemble_autotune(e, trial_blocks=0):
    d, s, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(load().sslbm_ensemble_autotune(e, int(trial_blocks), ctypes.byref(d), ctypes.byref(s),
                                          ctypes.byref(ms)), "sslbm_ensemble_autotune")
    return int(d.value), int(s.value), float(ms.value)


def sslbm_ensemble_steps_done(e):
    return int(load().sslbm_ensemble_steps_done(e))


def sslbm_ensemble_checkpoint_bytes(e) -> int:
    n = ctypes.c_size_t(0)
    _check(load().sslbm_ensemble_checkpoint_bytes(e, ctypes.byref(n)), "sslbm_ensemble_checkpoint_bytes")
    return int(n.value)


def sslbm_ensemble_checkpoint_save(e, dst):
    ptr, dev, nbytes = _raw(dst)
    _check(load().sslbm_ensemble_checkpoint_save(e, _vp(ptr), nbytes, dev), "sslbm_ensemble_checkpoint_save")
    return dst


def sslbm_ensemble_checkpoint_load(e, src):
    ptr, dev, nbytes = _raw(src)
    _check(load().sslbm_ensemble_checkpoint_load(e, _vp(ptr), nbytes, dev), "sslbm_ensemble_checkpoint_load")


# ---------------------------------------------------------------------------
# fourth-order finite-difference reference
# ---------------------------------------------------------------------------

def sslbm_fd4_workspace_bytes(g: Grid) -> int:
    n = ctypes.c_size_t(0)
    _check(load().sslbm_fd4_workspace_bytes(ctypes.byref(g), ctypes.byref(n)), "sslbm_fd4_workspace_bytes")
    return int(n.value)


def sslbm_fd4_create(g: Grid, p: Params, ws_ptr, ws_bytes, stream=0):
    f = _vp()
    _check(load().sslbm_fd4_create(ctypes.byref(g), ctypes.byref(p), _vp(ws_ptr), int(ws_bytes), _vp(stream),
                                   ctypes.byref(f)), "sslbm_fd4_create")
    return f


def sslbm_fd4_destroy(f):
    if f:
        load().sslbm_fd4_destroy(f)


def sslbm_fd4_write(f, src):
    ptr, dev, code, _ = _buffer(src)
    _check(load().sslbm_fd4_write(f, _vp(ptr), code, dev), "sslbm_fd4_write")


def sslbm_fd4_read(f, dst):
    ptr, dev, code, _ = _buffer(dst)
    _check(load().sslbm_fd4_read(f, _vp(ptr), code, dev), "sslbm_fd4_read")
    return dst


def sslbm_fd4_step(f, n):
    _check(load().sslbm_fd4_step(f, int(n)), "sslbm_fd4_step")


def sslbm_fd4_steps_done(f) -> int:
    return int(load().sslbm_fd4_steps_done(f))


def sslbm_fd4_set_order(f, order):
    _check(load().sslbm_fd4_set_order(f, int(order)), "sslbm_fd4_set_order")


class Fd4:
    """The fourth-order finite-difference reference (RK4 + fourth-order Laplacian) with a
    torch-allocated workspace; rates (beta, alpha, gamma, phi), d the physical
    diffusivities of S, E, I, R (and D = 0)."""

    def __init__(self, nx, ny, rates, d, dx=1.0, dt=1.0, bc=BC_PERIODIC, precision=FP64, order=4, device=None,
                 stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        self.grid = make_grid(nx, ny, dx, dt, bc, precision)
        self.params = make_params(*rates, d=d)
        self.nx, self.ny = int(nx), int(ny)
        nbytes = sslbm_fd4_workspace_bytes(self.grid)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.f = sslbm_fd4_create(self.grid, self.params, self.ws.data_ptr(), nbytes, self.stream.cuda_stream)
        sslbm_fd4_set_order(self.f, order)

    def close(self):
        if getattr(self, "f", None):
            self.stream.synchronize()
            sslbm_fd4_destroy(self.f)
            self.f = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def write(self, state):
        sslbm_fd4_write(self.f, state)

    def read(self, dtype=np.float64):
        return sslbm_fd4_read(self.f, np.empty((5, self.ny, self.nx), dtype=dtype))

    def step(self, n):
        sslbm_fd4_step(self.f, n)

    def steps_done(self):
        return sslbm_fd4_steps_done(self.f)


class Ensemble:
    """A batch of periodic scenarios with a torch-allocated device workspace."""

    def __init__(self, specs, precision=FP32, device=None, stream=None):
        import torch
        self.specs = list(specs)
        self.n = len(self.specs)
        self.precision = precision
        self.scen = make_scenarios(self.specs)
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = sslbm_ensemble_workspace_bytes(self.scen, precision)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.e = sslbm_ensemble_create(self.scen, precision, self.ws.data_ptr(), nbytes, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "e", None):
            self.stream.synchronize()
            sslbm_ensemble_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def write(self, idx, state):
        sslbm_ensemble_write(self.e, idx, state)

    def read(self, idx, dtype=np.float64):
        sp = self.specs[idx]
        out = np.empty((5, int(sp["ny"]), int(sp["nx"])), dtype=dtype)
        return sslbm_ensemble_read(self.e, idx, out)

    def run(self, nsteps):
        sslbm_ensemble_run(self.e, nsteps)

    def diagnostics(self):
        return sslbm_ensemble_diagnostics(self.e, self.n)

    def set_tiling(self, depth, seg_rows):
        sslbm_ensemble_set_tiling(self.e, depth, seg_rows)

    def get_tiling(self):
        return sslbm_ensemble_get_tiling(self.e)

    def checkpoint(self, on_device=False):
        """Every scenario's stored state and the step counter (host uint8 array, or a device
        tensor with on_device=True)."""
        n = sslbm_ensemble_checkpoint_bytes(self.e)
        if on_device:
            import torch
            buf = torch.empty(n, dtype=torch.uint8, device=self.device)
        else:
            buf = np.empty(n, dtype=np.uint8)
        return sslbm_ensemble_checkpoint_save(self.e, buf)

    def restore(self, buf):
        sslbm_ensemble_checkpoint_load(self.e, buf)

    def set_wait_limit(self, spin_limit, stall_item=-1):
        sslbm_ensemble_set_wait_limit(self.e, spin_limit, stall_item)

    def autotune(self, trial_blocks=0):
        return sslbm_ensemble_autotune(self.e, trial_blocks)


# ---------------------------------------------------------------------------
# learned surrogate
# ---------------------------------------------------------------------------

def _dptr(t):
    """Device pointer of a contiguous float32 CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return _vp(t.data_ptr())


def sslbm_fno_workspace_bytes(cfg: FnoConfig) -> int:
    n = ctypes.c_size_t(0)
    _check(load().sslbm_fno_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)), "sslbm_fno_workspace_bytes")
    return int(n.value)


def sslbm_fno_create(cfg, ws_ptr, ws_bytes, stream=0):
    f = _vp()
    _check(load().sslbm_fno_create(ctypes.byref(cfg), _vp(ws_ptr), int(ws_bytes), _vp(stream), ctypes.byref(f)),
           "sslbm_fno_create")
    return f


def sslbm_fno_destroy(f):
    if f:
        load().sslbm_fno_destroy(f)


def sslbm_fno_num_params(f) -> int:
    return int(load().sslbm_fno_num_params(f))


def sslbm_fno_set_params(f, theta):
    ptr, dev, code, _ = _buffer(theta)
    if code != DT_F32:
        raise TypeError("parameters are float32")
    _check(load().sslbm_fno_set_params(f, _vp(ptr), dev), "sslbm_fno_set_params")


def sslbm_fno_get_params(f, out):
    ptr, dev, code, _ = _buffer(out)
    _check(load().sslbm_fno_get_params(f, _vp(ptr), dev), "sslbm_fno_get_params")
    return out


def sslbm_fno_get_grads(f, out):
    ptr, dev, code, _ = _buffer(out)
    _check(load().sslbm_fno_get_grads(f, _vp(ptr), dev), "sslbm_fno_get_grads")
    return out


def sslbm_fno_make_input(f, batch, u, r0, logd, x):
    _check(load().sslbm_fno_make_input(f, int(batch), _dptr(u), _dptr(r0), _dptr(logd), _dptr(x)),
           "sslbm_fno_make_input")


def sslbm_fno_forward(f, batch, x, y):
    _check(load().sslbm_fno_forward(f, int(batch), _dptr(x), _dptr(y)), "sslbm_fno_forward")


def sslbm_fno_backward(f, batch, x, dy):
    _check(load().sslbm_fno_backward(f, int(batch), _dptr(x), _dptr(dy)), "sslbm_fno_backward")


def sslbm_fno_set_adam(f, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    _check(load().sslbm_fno_set_adam(f, beta1, beta2, eps, weight_decay), "sslbm_fno_set_adam")


def sslbm_fno_set_wait_limit(f, polls=0, stall=False):
    _check(load().sslbm_fno_set_wait_limit(f, int(polls), 1 if stall else 0), "sslbm_fno_set_wait_limit")


def sslbm_fno_set_loss_weights(f, mass_weight=0.0, neg_weight=0.0):
    _check(load().sslbm_fno_set_loss_weights(f, float(mass_weight), float(neg_weight)), "sslbm_fno_set_loss_weights")


def sslbm_fno_infer(f, batch, x, y):
    _check(load().sslbm_fno_infer(f, int(batch), _dptr(x), _dptr(y)), "sslbm_fno_infer")


def sslbm_fno_fused(f) -> bool:
    r = int(load().sslbm_fno_fused(f))
    _check(min(r, 0), "sslbm_fno_fused")
    return r == 1


def sslbm_fno_train_step(f, batch, x, target, y_scratch, dy_scratch, lr, want_loss=True):
    loss = ctypes.c_double(0.0)
    _check(load().sslbm_fno_train_step(f, int(batch), _dptr(x), _dptr(target), _dptr(y_scratch), _dptr(dy_scratch),
                                       float(lr), ctypes.byref(loss) if want_loss else None),
           "sslbm_fno_train_step")
    return float(loss.value) if want_loss else None


def sslbm_surrogate_rollout(f, e, batch, steps, k_steps, u, r0, logd, x_scratch, y_scratch,
                            mass_threshold=1e-4, neg_threshold=0.0, reach=0, want_residuals=True):
    """The C-ABI rollout (argument marshalling only): u (device, [batch, 5, n, n] float32) is
    advanced in place.  Returns (stats dict, residuals [steps, batch, 2] or None,
    fell_back [steps, batch] bool or None)."""
    res = np.empty((steps, batch, 2), np.float64) if want_residuals else None
    fb = np.empty((steps, batch), np.uint8) if want_residuals else None
    st = RolloutStats()
    _check(load().sslbm_surrogate_rollout(
        f, e, int(batch), int(steps), int(k_steps), _dptr(u), _dptr(r0), _dptr(logd), _dptr(x_scratch),
        _dptr(y_scratch), float(mass_threshold), float(neg_threshold), int(reach),
        res.ctypes.data_as(_vp) if res is not None else None, fb.ctypes.data_as(_vp) if fb is not None else None,
        ctypes.byref(st)), "sslbm_surrogate_rollout")
    stats = {k: getattr(st, k) for k, _ in RolloutStats._fields_}
    return stats, res, (fb.astype(bool) if fb is not None else None)


def sslbm_fno_check_project(f, batch, y, u, reach=0):
    res = (ctypes.c_double * (2 * batch))()
    _check(load().sslbm_fno_check_project(f, int(batch), _dptr(y), _dptr(u), int(reach), res),
           "sslbm_fno_check_project")
    return np.array(res[:]).reshape(batch, 2)


class Surrogate:
    """The learned surrogate with a torch-allocated workspace (see include/sslbm.h)."""

    def __init__(self, n=256, width=32, modes=12, layers=4, hidden=64, max_batch=16, device=None, stream=None):
        import torch
        self.torch = torch
        self.cfg = FnoConfig(int(n), int(width), int(modes), int(layers), int(hidden), int(max_batch))
        self.n, self.max_batch = int(n), int(max_batch)
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = sslbm_fno_workspace_bytes(self.cfg)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.f = sslbm_fno_create(self.cfg, self.ws.data_ptr(), nbytes, self.stream.cuda_stream)
        self.nparams = sslbm_fno_num_params(self.f)
        shape = (self.max_batch, 5, self.n, self.n)
        self._y = torch.empty(shape, dtype=torch.float32, device=self.device)
        self._dy = torch.empty(shape, dtype=torch.float32, device=self.device)

    def close(self):
        if getattr(self, "f", None):
            self.stream.synchronize()
            sslbm_fno_destroy(self.f)
            self.f = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        sslbm_fno_set_params(self.f, theta)

    def get_params(self):
        out = np.empty(self.nparams, dtype=np.float32)
        return sslbm_fno_get_params(self.f, out)

    def get_grads(self):
        out = np.empty(self.nparams, dtype=np.float32)
        return sslbm_fno_get_grads(self.f, out)

    def make_input(self, u, r0, logd):
        B = u.shape[0]
        x = self.torch.empty((B, 8, self.n, self.n), dtype=self.torch.float32, device=self.device)
        sslbm_fno_make_input(self.f, B, u, r0, logd, x)
        return x

    def forward(self, x, y=None):
        B = x.shape[0]
        if y is None:
            y = self.torch.empty((B, 5, self.n, self.n), dtype=self.torch.float32, device=self.device)
        sslbm_fno_forward(self.f, B, x, y)
        return y

    def backward(self, x, dy):
        sslbm_fno_backward(self.f, x.shape[0], x, dy)

    def set_loss_weights(self, mass_weight=0.0, neg_weight=0.0):
        sslbm_fno_set_loss_weights(self.f, mass_weight, neg_weight)

    def set_wait_limit(self, polls=0, stall=False):
        sslbm_fno_set_wait_limit(self.f, polls, stall)

    @property
    def fused(self):
        return sslbm_fno_fused(self.f)

    def infer(self, x, y=None):
        B = x.shape[0]
        if y is None:
            y = self.torch.empty((B, 5, self.n, self.n), dtype=self.torch.float32, device=self.device)
        sslbm_fno_infer(self.f, B, x, y)
        return y

    def train_step(self, x, target, lr, want_loss=True):
        B = x.shape[0]
        return sslbm_fno_train_step(self.f, B, x, target, self._y[:B], self._dy[:B], lr, want_loss)

    def check_project(self, y, u, reach=0):
        return sslbm_fno_check_project(self.f, y.shape[0], y, u, reach)
