"""ctypes binding of the C ABI declared in include/zernike_gb300.h (argument marshalling only).

Every computation happens in the CUDA library; this module only turns torch tensors into
device pointers, host mode lists into int32 arrays, and status codes into exceptions.
If the shared library has not been built the first call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

c_i32p = ctypes.POINTER(ctypes.c_int32)
c_dp = ctypes.c_void_p  # device pointers travel as void*

# name -> (restype, argtypes).  Must match include/zernike_gb300.h.
SIGNATURES = {
    "zp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "zp_last_error": (ctypes.c_char_p, []),
    "zp_version": (ctypes.c_int32, []),
    "zp_plan_create": (ctypes.c_int, [c_i32p, c_i32p, ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p)]),
    "zp_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "zp_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32)]),
    "zp_radial": (ctypes.c_int, [c_i32p, c_i32p, ctypes.c_int64, c_dp, ctypes.c_int64, ctypes.c_int32, c_dp, c_dp]),
    "zp_radial_plan": (ctypes.c_int, [ctypes.c_void_p, c_dp, ctypes.c_int64, ctypes.c_int32, c_dp, c_dp]),
    "zp_radial_plan_timed": (ctypes.c_int, [ctypes.c_void_p, c_dp, ctypes.c_int64, ctypes.c_int32, c_dp, c_dp,
                                            ctypes.POINTER(ctypes.c_float)]),
    "zp_basis": (ctypes.c_int, [c_i32p, c_i32p, ctypes.c_int64, c_dp, c_dp, ctypes.c_int64, ctypes.c_int32, c_dp, c_dp,
                                c_dp]),
    "zp_basis_plan": (ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, ctypes.c_int64, ctypes.c_int32, c_dp, c_dp, c_dp]),
    "zp_radial_per_mode": (ctypes.c_int, [ctypes.c_void_p, c_dp, ctypes.c_int64, c_dp, c_dp]),
    "zp_series_eval": (ctypes.c_int, [c_i32p, c_i32p, ctypes.c_int64, c_dp, c_dp, ctypes.c_int64, c_dp, ctypes.c_int64,
                                      ctypes.c_int, c_dp, c_dp]),
    "zp_series_eval_plan": (ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, ctypes.c_int64, c_dp, ctypes.c_int64,
                                           ctypes.c_int, c_dp, c_dp]),
    "zp_series_adjoint": (ctypes.c_int, [c_i32p, c_i32p, ctypes.c_int64, c_dp, c_dp, ctypes.c_int64, c_dp,
                                         ctypes.c_int64, c_dp, c_dp, c_dp, c_dp, c_dp]),
    "zp_device_wait_status": (ctypes.c_int, [ctypes.c_int32]),
    "zp_release_scratch": (ctypes.c_int, []),
    "zp_series_point_hessian": (ctypes.c_int, [c_i32p, c_i32p, ctypes.c_int64, c_dp, c_dp, ctypes.c_int64, c_dp,
                                               ctypes.c_int64, c_dp, c_dp, c_dp, c_dp, c_dp, c_dp, c_dp]),
    "zp_series_point_hessian_plan": (ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, ctypes.c_int64, c_dp, ctypes.c_int64,
                                                    c_dp, c_dp, c_dp, c_dp, c_dp, c_dp, c_dp]),
    "zp_series_point_hvp_plan": (ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, ctypes.c_int64, c_dp, ctypes.c_int64,
                                                c_dp, c_dp, c_dp, c_dp, c_dp, c_dp]),
    "zp_series_fit": (ctypes.c_int, [c_i32p, c_i32p, ctypes.c_int64, c_dp, c_dp, c_dp, ctypes.c_int64, c_dp,
                                     ctypes.c_int64, ctypes.c_double, c_dp, c_dp]),
    "zp_series_fit_plan": (ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, c_dp, ctypes.c_int64, c_dp, ctypes.c_int64,
                                          ctypes.c_double, c_dp, c_dp]),
    "zp_series_fit_plan_prec": (ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, c_dp, ctypes.c_int64, c_dp, ctypes.c_int64,
                                               ctypes.c_double, c_dp, ctypes.c_int, c_dp]),
    "zp_probe_fp64": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, c_dp, ctypes.POINTER(ctypes.c_double)]),
    "zp_device_wait_selftest": (ctypes.c_int, [ctypes.c_int32, c_dp]),
    "zp_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p)]),
    "zp_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "zp_batch_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_dp]),
    "zp_batch_forward_per_instance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_dp]),
    "zp_batch_adjoint": (ctypes.c_int, [ctypes.c_void_p, c_dp]),
    "zp_batch_adjoint_prec": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_dp]),
    "zp_batch_set_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32]),
    "zp_batch_get_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "zp_batch_tune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int, ctypes.c_int32, c_dp,
                                     ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]),
    "zp_series_eval_static": (ctypes.c_int, [c_i32p, c_i32p, ctypes.c_int64, c_dp, c_dp, ctypes.c_int64, c_dp,
                                             ctypes.c_int64, ctypes.c_int, c_dp, c_dp]),
    "zp_series_eval_timed": (ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, ctypes.c_int64, c_dp, ctypes.c_int64,
                                            ctypes.c_int, c_dp, c_dp, ctypes.POINTER(ctypes.c_float)]),
    "zp_series_adjoint_plan": (ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, ctypes.c_int64, c_dp, ctypes.c_int64, c_dp,
                                              c_dp, c_dp, c_dp, c_dp]),
    "zp_series_adjoint_plan_prec": (ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, ctypes.c_int64, c_dp, ctypes.c_int64,
                                                   c_dp, c_dp, c_dp, c_dp, ctypes.c_int, c_dp]),
}

_lib = None
_lock = threading.Lock()


class ZernikeError(RuntimeError):
    """A non-zero zp_status from the library."""

    def __init__(self, fn: str, status: int, message: str):
        super().__init__(f"{fn}: status {status} ({message})")
        self.status = status


def library_path() -> str:
    return _build.LIB_PATH


def load() -> ctypes.CDLL:
    """Load the shared library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing: run paper_2409_19156_gb300.build.build() "
                                   "(or __graft_entry__.build()) first; there is no CPU fallback")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(fn: str, status: int) -> None:
    if status != 0:
        lib = load()
        msg = lib.zp_status_string(status).decode()
        detail = lib.zp_last_error().decode()
        raise ZernikeError(fn, status, f"{msg}: {detail}" if detail else msg)


def call(fn: str, *args) -> None:
    check(fn, getattr(load(), fn)(*args))


def modes_i32(x) -> np.ndarray:
    """Host int32 contiguous copy of a mode list (list, numpy array or CPU tensor)."""
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x, dtype=np.int64).astype(np.int32))


def i32_ptr(a: np.ndarray):
    return a.ctypes.data_as(c_i32p)


class ZpInstance(ctypes.Structure):
    """Mirror of zp_instance (include/zernike_gb300.h)."""

    _fields_ = [("n", c_i32p), ("m", c_i32p), ("n_modes", ctypes.c_int64), ("r", ctypes.c_void_p),
                ("theta", ctypes.c_void_p), ("n_points", ctypes.c_int64), ("coeffs", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("grad_out", ctypes.c_void_p), ("grad_coeffs", ctypes.c_void_p),
                ("grad_r", ctypes.c_void_p), ("grad_theta", ctypes.c_void_p)]


def ptr(t) -> int | None:
    """Device pointer of a tensor (None for None)."""
    return None if t is None else t.data_ptr()
