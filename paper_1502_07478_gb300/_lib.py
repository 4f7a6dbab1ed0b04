"""ctypes declarations of the libtsp C ABI (include/tsp.h).

Argument marshalling only: every step of the reconstruction runs in the CUDA
library.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

TSP_OK = 0
TSP_EINVAL = -1
TSP_ENOMEM = -2
TSP_ECUDA = -3
TSP_ETIMEOUT = -4
TSP_ESTATE = -5

_ERR_NAMES = {TSP_EINVAL: "TSP_EINVAL", TSP_ENOMEM: "TSP_ENOMEM", TSP_ECUDA: "TSP_ECUDA",
              TSP_ETIMEOUT: "TSP_ETIMEOUT", TSP_ESTATE: "TSP_ESTATE"}


class TspError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("R", C.c_double), ("L", C.c_double), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dy", C.c_double), ("dz", C.c_double), ("sigma_z", C.c_double),
                ("sigma_dl", C.c_double), ("cut", C.c_double), ("flags", C.c_int32),
                ("reserved", C.c_int32), ("gamma", C.c_double), ("kappa_z", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("n_events", C.c_int64), ("n_used", C.c_int64), ("n_empty", C.c_int64),
                ("n_outliers", C.c_int64), ("n_window", C.c_int64), ("iterations", C.c_int64),
                ("launches", C.c_int64), ("n_qbad", C.c_int64), ("n_clipped", C.c_int64),
                ("sum_s_rho", C.c_double), ("dbg_violation", C.c_int64)]


class Schedule(C.Structure):
    _fields_ = [("ty_cap", C.c_int32), ("items_per_sm", C.c_int32), ("order", C.c_int32),
                ("reserved", C.c_int32)]


# (name, restype, argtypes) of every exported entry point
_vp = C.c_void_p
_fp = C.c_void_p          # float* (host or device address)
SIGNATURES = [
    ("tsp_create", C.c_int, [C.POINTER(Params), C.POINTER(_vp)]),
    ("tsp_destroy", None, [_vp]),
    ("tsp_last_error", C.c_char_p, [_vp]),
    ("tsp_version", C.c_char_p, []),
    ("tsp_upload_events", C.c_int, [_vp, _fp, _fp, _fp, C.c_int64, C.c_int, _vp]),
    ("tsp_begin_events", C.c_int, [_vp, C.c_int64, _vp]),
    ("tsp_append_events", C.c_int, [_vp, _fp, _fp, _fp, C.c_int64, C.c_int, _vp]),
    ("tsp_end_events", C.c_int, [_vp, _vp]),
    ("tsp_compute_sensitivity", C.c_int, [_vp, _fp, C.c_int, _vp]),
    ("tsp_set_image", C.c_int, [_vp, _fp, C.c_int, _vp]),
    ("tsp_iterate", C.c_int, [_vp, C.c_int, _vp]),
    ("tsp_read_image", C.c_int, [_vp, _fp, C.c_int, C.c_int, _vp]),
    ("tsp_direct_image", C.c_int, [_vp, _fp, C.c_int, _vp]),
    ("tsp_backproject", C.c_int, [_vp, _fp, C.c_int, _vp]),
    ("tsp_apply_update", C.c_int, [_vp, _fp, C.c_int, _vp]),
    ("tsp_wait", C.c_int, [_vp, _vp, C.c_int]),
    ("tsp_loglik", C.c_int, [_vp, C.POINTER(C.c_double), _vp]),
    ("tsp_loglik_grad", C.c_int, [_vp, C.POINTER(C.c_double), _fp, C.c_int,
                                  C.POINTER(C.c_double), _vp]),
    ("tsp_set_sigma", C.c_int, [_vp, C.c_double, C.c_double, _vp]),
    ("tsp_stats", C.c_int, [_vp, C.POINTER(Stats), _vp]),
    ("tsp_set_profiling", C.c_int, [_vp, C.c_int]),
    ("tsp_pass_times", C.c_int, [_vp, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int), _vp]),
    ("tsp_set_variant", C.c_int, [_vp, C.c_int]),
    ("tsp_get_schedule", C.c_int, [_vp, C.POINTER(Schedule)]),
    ("tsp_set_schedule", C.c_int, [_vp, C.POINTER(Schedule), _vp]),
    ("tsp_autotune", C.c_int, [_vp, C.POINTER(Schedule), C.POINTER(C.c_float), _vp]),
    ("tsp_batch_create", C.c_int, [C.POINTER(Params), C.c_int, C.POINTER(_vp)]),
    ("tsp_batch_destroy", None, [_vp]),
    ("tsp_batch_last_error", C.c_char_p, [_vp]),
    ("tsp_batch_size", C.c_int, [_vp]),
    ("tsp_batch_upload_events", C.c_int, [_vp, C.c_int, _fp, _fp, _fp, C.c_int64, C.c_int, _vp]),
    ("tsp_batch_set_image", C.c_int, [_vp, C.c_int, _fp, C.c_int, _vp]),
    ("tsp_batch_set_sigma", C.c_int, [_vp, C.c_int, C.c_double, C.c_double, _vp]),
    ("tsp_batch_iterate", C.c_int, [_vp, C.c_int, _vp]),
    ("tsp_batch_read_image", C.c_int, [_vp, C.c_int, _fp, C.c_int, C.c_int, _vp]),
    ("tsp_batch_loglik_grad", C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double), _vp]),
    ("tsp_batch_stats", C.c_int, [_vp, C.c_int, C.POINTER(Stats), _vp]),
    ("tsp_batch_get_schedule", C.c_int, [_vp, C.POINTER(Schedule)]),
    ("tsp_batch_set_schedule", C.c_int, [_vp, C.POINTER(Schedule), _vp]),
    ("tsp_batch_autotune", C.c_int, [_vp, C.POINTER(Schedule), C.POINTER(C.c_float), _vp]),
    ("tsp_batch_set_profiling", C.c_int, [_vp, C.c_int]),
    ("tsp_batch_pass_times", C.c_int, [_vp, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int),
                                       _vp]),
    ("tsp_mlem_update_noalloc", C.c_int, [C.POINTER(Params), _fp, _fp, _fp, C.c_int64, _fp, _fp,
                                          _fp, _vp, C.c_char_p, C.c_size_t]),
]

_lib = None


def lib():
    """The loaded libtsp (raises if it has not been built).  The environment
    variable TSP_LIBRARY names another build of it to load instead (the
    bounds-checking build of ``build(debug=True)``)."""
    global _lib
    if _lib is None:
        path = os.environ.get("TSP_LIBRARY") or LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libtsp is not built ({path} missing); run "
                               "`python -m paper_1502_07478_gb300.build` or "
                               "`__graft_entry__.build()` first")
        L = C.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(ctx, rc: int):
    if rc != TSP_OK:
        msg = lib().tsp_last_error(ctx)
        raise TspError(rc, msg.decode() if msg else "")


def check_batch(batch, rc: int):
    if rc != TSP_OK:
        msg = lib().tsp_batch_last_error(batch)
        raise TspError(rc, msg.decode() if msg else "")
