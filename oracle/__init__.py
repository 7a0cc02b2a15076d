"""FP64 CPU oracle for Fuzzy C-Means — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never calls it and
shares no code with it; the two meet only in the seeded inputs of the
``phantom`` module.

``fcm_oracle.c`` holds the plain definitions (Eq. 1, 3, 4 and Algorithm 1 of
arXiv:1601.00072) in FP64; this module compiles it with gcc and wraps it with
ctypes. ``mlp`` holds the FP64 forward/backward of the warm-start network.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(hand-computed rationals, closed forms, optimality properties, special cases,
metamorphic relations, planted-mistake checks); see ``tests/test_oracle*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fcm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_fcm.so")
_lock = threading.Lock()
_lib = None

CONVERGED = 0
NOT_CONVERGED = 1
INIT_U = 0
INIT_V = 1

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i = ctypes.POINTER(ctypes.c_int)
_u8 = ctypes.POINTER(ctypes.c_uint8)


def build(src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle into a shared library (plain C, -O2, IEEE FP64)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (os.path.exists(out) and src == _SRC
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def _bind(lib):
    lib.oracle_memberships.argtypes = [_d, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_double, _d, _d]
    lib.oracle_memberships.restype = None
    lib.oracle_centers.argtypes = [_d, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_double, _d, _d, _d, _d, _d]
    lib.oracle_centers.restype = ctypes.c_int
    lib.oracle_objective.argtypes = [_d, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_double, _d, _d]
    lib.oracle_objective.restype = ctypes.c_double
    lib.oracle_labels.argtypes = [_d, ctypes.c_int64, ctypes.c_int, _i32]
    lib.oracle_labels.restype = None
    common = [ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
              ctypes.c_int, ctypes.c_int, _d, _d, _d, _i, _d, _d, _d, _i]
    lib.oracle_fcm.argtypes = [_d] + common
    lib.oracle_fcm.restype = ctypes.c_int
    lib.oracle_fcm_quantized.argtypes = [_u8] + common
    lib.oracle_fcm_quantized.restype = ctypes.c_int
    if hasattr(lib, "oracle_fcm_multi"):
        lib.oracle_memberships_multi.argtypes = [_d, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_double, _d, _d]
        lib.oracle_memberships_multi.restype = None
        lib.oracle_objective_multi.argtypes = [_d, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_double, _d, _d]
        lib.oracle_objective_multi.restype = ctypes.c_double
        lib.oracle_fcm_multi.argtypes = [_d, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, _d, _d, _d, _i, _d,
                                         _d, _i]
        lib.oracle_fcm_multi.restype = ctypes.c_int
    if hasattr(lib, "oracle_dsc"):
        lib.oracle_dsc.argtypes = [_i32, _u8, ctypes.c_int64, _i32, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int64), _d]
        lib.oracle_dsc.restype = ctypes.c_int
    return lib


def load_library(path: str):
    """Load an oracle library built from ``fcm_oracle.c`` (or a variant)."""
    return _bind(ctypes.CDLL(path))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
        return _lib


def _p(a, t=_d):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def memberships(x, V, m, L=None):
    """Eq. 4 (with the zero-distance rule): U [C, n] in FP64."""
    L = L or lib()
    x, V = _f64(x).reshape(-1), _f64(V).reshape(-1)
    if not 1 <= V.size <= 64:
        raise ValueError("C must be in [1, 64]")
    U = np.empty((V.size, x.size))
    L.oracle_memberships(_p(x), x.size, V.size, float(m), _p(V), _p(U))
    return U


def centers(x, U, m, Vprev=None, L=None):
    """Eq. 3: returns (V, num, den, n_empty)."""
    L = L or lib()
    x, U = _f64(x).reshape(-1), _f64(U)
    C = U.shape[0]
    V, num, den = np.empty(C), np.empty(C), np.empty(C)
    vp = None if Vprev is None else _f64(Vprev)
    e = L.oracle_centers(_p(x), x.size, C, float(m), _p(U), _p(vp), _p(V),
                         _p(num), _p(den))
    return V, num, den, e


def objective(x, U, V, m, L=None):
    """Eq. 1: J_m(U, V)."""
    L = L or lib()
    x, U, V = _f64(x).reshape(-1), _f64(U), _f64(V)
    return L.oracle_objective(_p(x), x.size, U.shape[0], float(m), _p(U), _p(V))


def labels(U, L=None):
    """Defuzzification: argmax over clusters, ties to the lowest index."""
    L = L or lib()
    U = _f64(U)
    out = np.empty(U.shape[1], dtype=np.int32)
    L.oracle_labels(_p(U), U.shape[1], U.shape[0], _p(out, _i32))
    return out


def memberships_multi(x, V, m, L=None):
    """Eq. 4 with the Euclidean norm over D channels: x [D, n], V [C, D]."""
    L = L or lib()
    x = _f64(x)
    V = _f64(V)
    D, n = x.shape
    U = np.empty((V.shape[0], n))
    L.oracle_memberships_multi(_p(x), n, D, V.shape[0], float(m), _p(V), _p(U))
    return U


def objective_multi(x, U, V, m, L=None):
    L = L or lib()
    x, U, V = _f64(x), _f64(U), _f64(V)
    return L.oracle_objective_multi(_p(x), x.shape[1], x.shape[0], V.shape[0], float(m), _p(U), _p(V))


def fcm_multi(x, C, m, eps, max_iter, U0=None, V0=None, want_U=True, L=None):
    """Algorithm 1 on D-channel pixels: x [D, n]; give U0 [C, n] or V0 [C, D].
    Returns U, V [C, D], iters, status, delta/J traces, empty."""
    L = L or lib()
    x = _f64(x)
    D, n = x.shape
    if (U0 is None) == (V0 is None):
        raise ValueError("give exactly one of U0 and V0")
    mode, init = (INIT_U, _f64(U0).reshape(C, n)) if U0 is not None else (INIT_V, _f64(V0).reshape(C, D))
    U = np.empty((C, n)) if want_U else None
    V = np.empty((C, D))
    iters, empty = ctypes.c_int(0), ctypes.c_int(0)
    td, tJ = np.zeros(max_iter), np.zeros(max_iter)
    st = L.oracle_fcm_multi(_p(x), n, D, C, float(m), float(eps), int(max_iter), mode, _p(init), _p(U), _p(V),
                            ctypes.byref(iters), _p(td), _p(tJ), ctypes.byref(empty))
    if st < 0:
        raise ValueError(f"oracle rejected the arguments (status {st})")
    k = iters.value
    return {"U": U, "V": V, "iters": k, "status": st, "delta": td[:k], "J": tJ[:k], "empty": empty.value}


def dsc(labels_, truth, class_of_label, n_classes, L=None):
    """Dice similarity per class (Sec. 5.2, Eq. 5) of labels (mapped to
    classes by class_of_label) against truth. Returns (dsc [n_classes],
    counts [n_classes, 3] of |PR|, |GT|, |PR n GT|)."""
    L = L or lib()
    lab = np.ascontiguousarray(labels_, dtype=np.int32).reshape(-1)
    tr = np.ascontiguousarray(truth, dtype=np.uint8).reshape(-1)
    cl = np.ascontiguousarray(class_of_label, dtype=np.int32).reshape(-1)
    out = np.empty(n_classes)
    counts = np.empty(3 * n_classes, dtype=np.int64)
    st = L.oracle_dsc(_p(lab, _i32), _p(tr, _u8), lab.size, _p(cl, _i32), cl.size, n_classes,
                      counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _p(out))
    if st < 0:
        raise ValueError("oracle rejected the arguments")
    return out, counts.reshape(n_classes, 3)


def _run(fn, xarg, n, C, m, eps, max_iter, U0, V0, want_U):
    if (U0 is None) == (V0 is None):
        raise ValueError("give exactly one of U0 and V0")
    if U0 is not None:
        mode, init = INIT_U, _f64(U0).reshape(C, n)
    else:
        mode, init = INIT_V, _f64(V0).reshape(C)
    U = np.empty((C, n)) if want_U else None
    V = np.empty(C)
    iters = ctypes.c_int(0)
    empty = ctypes.c_int(0)
    td, tJ = np.zeros(max_iter), np.zeros(max_iter)
    tV = np.zeros((max_iter, C))
    st = fn(xarg, n, C, float(m), float(eps), int(max_iter), mode, _p(init),
            _p(U), _p(V), ctypes.byref(iters), _p(td), _p(tJ), _p(tV),
            ctypes.byref(empty))
    if st < 0:
        raise ValueError(f"oracle rejected the arguments (status {st})")
    k = iters.value
    return {"U": U, "V": V, "iters": k, "status": st, "delta": td[:k],
            "J": tJ[:k], "Vtrace": tV[:k], "empty": empty.value}


def fcm(x, C, m, eps, max_iter, U0=None, V0=None, want_U=True, L=None):
    """Algorithm 1 on every pixel, FP64. Give U0 [C, n] or V0 [C].

    Returns a dict: U (final memberships, or None), V, iters, status
    (CONVERGED / NOT_CONVERGED), delta/J/Vtrace per iteration, empty.
    """
    L = L or lib()
    x = _f64(x).reshape(-1)
    return _run(L.oracle_fcm, _p(x), x.size, C, m, eps, max_iter, U0, V0, want_U)


def fcm_quantized(xq, C, m, eps, max_iter, U0=None, V0=None, want_U=False, L=None):
    """Algorithm 1 for uint8 grey levels, run on the 256-bin histogram."""
    L = L or lib()
    xq = np.ascontiguousarray(xq, dtype=np.uint8).reshape(-1)
    return _run(L.oracle_fcm_quantized, _p(xq, _u8), xq.size, C, m, eps,
                max_iter, U0, V0, want_U)
