"""ctypes declarations of the C ABI in ``include/fcm.h``.

Loading fails loudly when the library has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

FCM_MAX_CLUSTERS = 8
FCM_OK = 0
FCM_NOT_CONVERGED = 1
FCM_ERR_INVALID_ARG = -1
FCM_ERR_CUDA = -2
FCM_ERR_OOM = -3
FCM_ERR_BAD_INPUT = -4
FCM_ERR_NONFINITE = FCM_ERR_BAD_INPUT
FCM_ERR_TIMEOUT = -5
FCM_ERR_TOO_LARGE = -6
FCM_NOALLOC_MAX_BLOCKS = 512
FCM_FLAG_EMPTY_CLUSTER = 1
FCM_FLAG_BOUNDS = 2
FCM_INIT_U = 0
FCM_INIT_V = 1
FCM_OPT_TRACE = 1
FCM_OPT_NO_GRAPH = 2
FCM_OPT_NO_TMA = 4
FCM_OPT_NO_PERSISTENT = 8
FCM_OPT_RECOMPUTE = 16
FCM_OPT_DETERMINISTIC = 32


class fcm_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("flags", ctypes.c_int),
                ("C", ctypes.c_int), ("delta", ctypes.c_double), ("J", ctypes.c_double),
                ("V64", ctypes.c_double * FCM_MAX_CLUSTERS), ("launches", ctypes.c_int),
                ("reserved", ctypes.c_int)]


class fcm_slice(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("n", ctypes.c_int64), ("C", ctypes.c_int),
                ("m", ctypes.c_float), ("eps", ctypes.c_float), ("max_iter", ctypes.c_int),
                ("init_mode", ctypes.c_int), ("iters_hint", ctypes.c_int),
                ("U0", ctypes.c_void_p), ("U", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("V0", ctypes.c_float * FCM_MAX_CLUSTERS),
                ("iters", ctypes.c_int), ("status", ctypes.c_int), ("flags", ctypes.c_int),
                ("reserved1", ctypes.c_int), ("delta", ctypes.c_double), ("J", ctypes.c_double),
                ("V64", ctypes.c_double * FCM_MAX_CLUSTERS)]


class fcm_limits(ctypes.Structure):
    _fields_ = [("grid_wait_spins", ctypes.c_uint32), ("tma_wait_polls", ctypes.c_uint32),
                ("barrier_phantoms", ctypes.c_uint32), ("fail_alloc_in", ctypes.c_int32)]


class fcm_batch_plan(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("cluster", ctypes.c_int), ("big", ctypes.c_int64),
                ("ms", ctypes.c_double), ("schedule", ctypes.c_int), ("tile", ctypes.c_int)]


FCM_SCHED_SLICES = 0
FCM_SCHED_ROUNDS = 1
FCM_SCHED_TEAMS = 2


FCM_BATCH_RETUNE = 16
FCM_BATCH_NO_TUNE = 32
FCM_BATCH_NO_GRAPH = 64
FCM_BATCH_PRESOLVE = 128
FCM_MODEL_PARAMS = 51464
MODEL_D_IN = 264
MODEL_D_OUT = 8

_vp = ctypes.c_void_p
_i = ctypes.c_int
_f = ctypes.c_float
_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)

# (name, restype, argtypes) of every entry point declared in include/fcm.h
SIGNATURES = [
    ("fcm_create", _i, [ctypes.POINTER(_vp), _i, _vp]),
    ("fcm_set_stream", _i, [_vp, _vp]),
    ("fcm_destroy", None, [_vp]),
    ("fcm_set_limits", _i, [_vp, ctypes.POINTER(fcm_limits)]),
    ("fcm_get_limits", _i, [_vp, ctypes.POINTER(fcm_limits)]),
    ("fcm_run", _i, [_vp, _vp, _i64, _i, _f, _f, _i, _i, _vp, _vp, _vp, _i,
                     ctypes.POINTER(fcm_report)]),
    ("fcm_init_dirichlet", _i, [_vp, _i64, _i, ctypes.c_uint64, _vp]),
    ("fcm_run_seeded", _i, [_vp, _vp, _i64, _i, _f, _f, _i, ctypes.c_uint64, _vp, _vp, _i,
                            ctypes.POINTER(fcm_report)]),
    ("fcm_run_stream", _i, [_vp, _i, ctypes.POINTER(_vp), _i64, _i, _f, _f, _i, ctypes.POINTER(_vp),
                            ctypes.POINTER(_vp), _vp, _i, ctypes.POINTER(fcm_report)]),
    ("fcm_run_hist", _i, [_vp, _vp, _i64, _i, _f, _f, _i, _i, _vp, _vp, _vp, ctypes.POINTER(fcm_report)]),
    ("fcm_dsc", _i, [_vp, _vp, _i64, _i, _vp, ctypes.POINTER(_i), _i, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double)]),
    ("fcm_run_multi", _i, [_vp, _vp, _i64, _i, _i, _f, _f, _i, _i, _vp, _vp, _vp,
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(fcm_report)]),
    ("fcm_run_batched", _i, [_vp, ctypes.POINTER(fcm_slice), _i, _i]),
    ("fcm_run_batched_hist", _i, [_vp, ctypes.POINTER(fcm_slice), _i]),
    ("fcm_batched_plan", _i, [_vp, ctypes.POINTER(fcm_batch_plan)]),
    ("fcm_batched_set_plan", _i, [_vp, ctypes.POINTER(fcm_batch_plan)]),
    ("fcm_model_init", _i, [_vp, ctypes.c_uint64]),
    ("fcm_model_set_params", _i, [_vp, ctypes.POINTER(_f), _i64]),
    ("fcm_model_get_params", _i, [_vp, ctypes.POINTER(_f), _i64]),
    ("fcm_model_save", _i, [_vp, ctypes.c_char_p]),
    ("fcm_model_load", _i, [_vp, ctypes.c_char_p]),
    ("fcm_features", _i, [_vp, ctypes.POINTER(fcm_slice), _i, _vp]),
    ("fcm_model_forward", _i, [_vp, _vp, _i, _vp]),
    ("fcm_model_loss_grad", _i, [_vp, _vp, _vp, _vp, _i, ctypes.POINTER(_f), ctypes.POINTER(_f)]),
    ("fcm_model_train", _i, [_vp, _vp, _vp, _vp, _i, _i, _i, _f, ctypes.c_uint64, ctypes.POINTER(_f)]),
    ("fcm_predict_centers", _i, [_vp, ctypes.POINTER(fcm_slice), _i]),
    ("fcm_run_batched_warm", _i, [_vp, ctypes.POINTER(fcm_slice), _i, _i, ctypes.POINTER(_i)]),
    ("fcm_run_noalloc", _i, [_vp, _i64, _i, _f, _f, _i, _i, _vp, _vp, _vp, _vp,
                             ctypes.POINTER(fcm_report)]),
    ("fcm_time_pass", _i, [_vp, _vp, _i64, _i, _f, _vp, _vp, _i, _i, ctypes.POINTER(_f)]),
    ("fcm_get_trace", _i, [_vp, _dp, _dp, _dp, _i]),
    ("fcm_last_error", ctypes.c_char_p, [_vp]),
    ("fcm_status_string", ctypes.c_char_p, [_i]),
    ("fcm_version", ctypes.c_char_p, []),
]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load ``libfcm_gb300.so`` and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(
                f"the FCM CUDA library is not built ({path} missing); "
                "run `python -c 'import __graft_entry__ as g; g.build()'` first")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FcmError(RuntimeError):
    def __init__(self, status: int, message: str = ""):
        self.status = status
        name = load().fcm_status_string(status).decode()
        super().__init__(f"{name} ({status})" + (f": {message}" if message else ""))


def check(status: int, handle=None) -> int:
    if status < 0:
        msg = ""
        if handle is not None:
            raw = load().fcm_last_error(handle)
            msg = raw.decode() if raw else ""
        raise FcmError(status, msg)
    return status
