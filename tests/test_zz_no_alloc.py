"""fcm_run_noalloc gives the same segmentation as fcm_run (needs a GPU).

fcm_run_noalloc is for callers that cannot allocate device memory while they
run — memory owned by a pool or a framework allocator, plugins that are handed
only pre-allocated buffers, latency-critical services that cannot afford a
cudaMalloc. It keeps its scratch in a fixed device array inside the library
instead of a handle's workspace. This file is collected after every other test
file, so a run that stops at its first failure has already run the rest; it
also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import phantom
from parity import U_TOL, center_err

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_fcm_run_on_two_calls_in_a_row():
    import torch

    from paper_1601_00072_gb300 import _build, _lib
    _build.build()
    L = _lib.load()
    x, _, u0, C = phantom.single_image("phantom200")
    n = x.size
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    xd = torch.from_numpy(x.astype(np.float32)).to(dev)
    U0 = torch.from_numpy(u0).to(dev)

    # the existing entry point, through the C ABI, as the reference
    h = ctypes.c_void_p()
    assert L.fcm_create(ctypes.byref(h), 0, None) == 0
    try:
        Uref = torch.empty_like(U0)
        Vref = torch.empty(C, dtype=torch.float32, device=dev)
        rep_ref = _lib.fcm_report()
        st_ref = L.fcm_run(h, _p(xd), n, C, 2.0, 1e-5, 300, _lib.FCM_INIT_U, _p(U0), _p(Uref),
                           _p(Vref), 0, ctypes.byref(rep_ref))
        assert st_ref == _lib.FCM_OK
    finally:
        L.fcm_destroy(h)
    Uref, Vref = Uref.cpu().numpy(), Vref.cpu().numpy()

    for call in range(2):
        U = torch.full_like(U0, -1.0)
        V = torch.full((C,), -1.0, dtype=torch.float32, device=dev)
        rep = _lib.fcm_report()
        st = L.fcm_run_noalloc(_p(xd), n, C, 2.0, 1e-5, 300, _lib.FCM_INIT_U, _p(U0), _p(U), _p(V),
                               None, ctypes.byref(rep))
        assert st == _lib.FCM_OK, (call, st)
        assert rep.iters == rep_ref.iters, (call, rep.iters, rep_ref.iters)
        assert np.max(np.abs(U.cpu().numpy() - Uref)) <= U_TOL, call
        assert center_err(V.cpu().numpy(), Vref) <= 1e-5, call
        assert np.array_equal(U0.cpu().numpy(), u0)  # the initial membership is only read

    # shapes it cannot take without staging (and so without allocating)
    assert L.fcm_run_noalloc(_p(xd), n - 1, C, 2.0, 1e-5, 300, _lib.FCM_INIT_U, _p(U0), _p(U), _p(V),
                             None, None) == _lib.FCM_ERR_INVALID_ARG
    xh = np.ascontiguousarray(x.astype(np.float32))
    assert L.fcm_run_noalloc(ctypes.c_void_p(xh.ctypes.data), n, C, 2.0, 1e-5, 300, _lib.FCM_INIT_U,
                             _p(U0), _p(U), _p(V), None, None) == _lib.FCM_ERR_INVALID_ARG
