"""Loader of the in-tree CUDA library libdracogb.so (ctypes).

There is no fallback: if the library is missing or cannot be loaded, every
call raises.  Build it with `paper_2410_14900_gb300.build.build()` (or
`__graft_entry__.build()`).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

(DC_OK, DC_ERR_ARG, DC_ERR_CUDA, DC_ERR_OOM, DC_ERR_TIMEOUT, DC_ERR_UNSUPPORTED,
 DC_ERR_NONFINITE) = range(7)
DC_F32, DC_BF16, DC_F16, DC_F32X2 = 0, 1, 2, 3
DC_ACCUM, DC_KAHAN, DC_RELU = 1, 2, 4
DC_PERSISTENT_FILTER = 8
DC_VIEW_GEO_N = 24


class dc_geometry_desc(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int), ("det_rows", ctypes.c_int),
                ("det_cols", ctypes.c_int), ("n_mu", ctypes.c_int), ("n_s", ctypes.c_int),
                ("pitch", ctypes.c_double), ("ds", ctypes.c_double),
                ("vol_x", ctypes.c_int), ("vol_y", ctypes.c_int), ("vol_z", ctypes.c_int),
                ("voxel", ctypes.c_double * 3), ("vol_center", ctypes.c_double * 3),
                ("closed_orbit", ctypes.c_int)]


class DCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} [status {code}]")
        self.code = code


_P = ctypes.c_void_p
_SIGS = {
    "dc_setup_geometry": (ctypes.c_int, [ctypes.POINTER(dc_geometry_desc), _P, _P,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "dc_destroy_geometry": (None, [_P]),
    "dc_get_view_geometry": (ctypes.c_int, [_P, _P]),
    "dc_filter": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, _P]),
    "dc_filter_adjoint": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, ctypes.c_int,
                                         _P]),
    "dc_backproject": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, _P, _P,
                                      ctypes.c_uint, _P]),
    "dc_backproject_adjoint": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P]),
    "dc_grangeat": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "dc_radon2d": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "dc_radon2d_adjoint": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "dc_sync_status": (ctypes.c_int, [_P, _P]),
    "dc_crofton_weights": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int,
                                          _P, _P]),
    "dc_reconstruct_host": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, ctypes.c_int, _P, _P,
                                           _P, ctypes.c_uint, ctypes.c_int, _P]),
    "dc_microbench": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
    "dc_gauss_smooth": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                       ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "dc_batch_create": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_int, ctypes.c_uint,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "dc_batch_run": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "dc_batch_set_bp_nz": (ctypes.c_int, [_P, ctypes.c_int]),
    "dc_batch_destroy": (None, [_P]),
    "dc_geometry_set_tuning": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "dc_geometry_get_tuning": (ctypes.c_int, [_P, _P, _P, _P]),
    "dc_radon2d_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, _P, _P, _P]),
    "dc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "dc_last_error": (ctypes.c_char_p, []),
    "dc_version": (ctypes.c_char_p, []),
    "dc_launch_count": (ctypes.c_ulonglong, []),
    "dc_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "dc_profile_collect": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "dc_profile_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
    "dc_debug_fail_alloc_after": (None, [ctypes.c_long]),
    "dc_debug_wait_timeout": (ctypes.c_int, [_P, _P]),
    "dc_deriv": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "dc_filter_with_s": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, _P, _P]),
    "dc_filter_adjoint_from_s": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P,
                                                ctypes.c_int, _P]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libdracogb.so (raising if it is absent and not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run "
                               "paper_2410_14900_gb300.build.build() first")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def check(rc: int, what: str):
    if rc != DC_OK:
        L = load()
        msg = L.dc_last_error().decode() or L.dc_status_string(rc).decode()
        raise DCError(rc, f"{what}: {msg}")
