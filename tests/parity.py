"""Comparison of a CUDA FCM result with the FP64 oracle.

Thresholds (stated for every result):
  center error     |v_gpu - v_ref| / max(|v_ref|, 1)  <= 1e-5
  memberships      max |u_gpu - u_ref|                 <= 1e-5
  labels           argmax agreement                    >= 99.99 %
  iterations       |k_gpu - k_ref|                     <= 1
The max(|v|, 1) denominator keeps the relative error of a center near 0 (the
background class) meaningful. When the iteration counts differ by one, U and V
are compared at the common iteration count (the longer run is repeated with
max_iter set to it), so the comparison is always between the same iterate.
"""
from __future__ import annotations

import numpy as np

CENTER_TOL = 1e-5
U_TOL = 1e-5
LABEL_AGREE = 0.9999
ITER_TOL = 1


def eps32(eps: float) -> float:
    """The FP32 value the CUDA path compares against, as a double."""
    return float(np.float32(eps))


def center_err(v, ref) -> float:
    v, ref = np.asarray(v, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(v - ref) / np.maximum(np.abs(ref), 1.0)))


def labels_of(U) -> np.ndarray:
    U = np.asarray(U)
    return np.argmax(U, axis=0)  # ties to the lowest index


def precision_report(gpu_U, gpu_V, gpu_iters, ref_U, ref_V, ref_iters, gpu_J=None, ref_J=None):
    """Errors of a CUDA result against the oracle (U may be a sample)."""
    gU = np.asarray(gpu_U, dtype=np.float64)
    rU = np.asarray(ref_U, dtype=np.float64)
    rep = {
        "center_rel_err": center_err(gpu_V, ref_V),
        "max_abs_dU": float(np.max(np.abs(gU - rU))),
        "label_agreement": float(np.mean(labels_of(gU) == labels_of(rU))),
        "d_iters": int(gpu_iters) - int(ref_iters),
    }
    if gpu_J is not None and ref_J is not None:
        rep["J_rel_err"] = float(abs(gpu_J - ref_J) / max(abs(ref_J), 1e-300))
    return rep


def assert_within(rep, iters_checked=True):
    msgs = []
    if rep["center_rel_err"] > CENTER_TOL:
        msgs.append(f"center rel err {rep['center_rel_err']:.3g} > {CENTER_TOL}")
    if rep["max_abs_dU"] > U_TOL:
        msgs.append(f"max|dU| {rep['max_abs_dU']:.3g} > {U_TOL}")
    if rep["label_agreement"] < LABEL_AGREE:
        msgs.append(f"label agreement {rep['label_agreement']:.6f} < {LABEL_AGREE}")
    if iters_checked and abs(rep["d_iters"]) > ITER_TOL:
        msgs.append(f"iteration count differs by {rep['d_iters']}")
    assert not msgs, "; ".join(msgs) + f"  ({rep})"
