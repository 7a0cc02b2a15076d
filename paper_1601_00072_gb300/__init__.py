"""GB300 Fuzzy C-Means image segmentation (arXiv:1601.00072) behind a C ABI.

The CUDA library ``libfcm_gb300.so`` (sources in ``csrc/``, ABI in
``include/fcm.h``) runs the per-iteration pixel pass; this package builds it
(``_build``), declares its entry points (``_lib``) and wraps them for torch
tensors (``fcm``). There is no CPU fallback.
"""
from ._lib import FcmError, load  # noqa: F401


def __getattr__(name):
    if name in ("FCM", "FCMResult"):
        from . import fcm
        return getattr(fcm, name)
    raise AttributeError(name)
