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


def test_noalloc_allocates_nothing_and_takes_host_centers():
    """After one warm-up call per kernel (the first call on a device resolves
    the scratch address, and the driver loads each kernel's module on its
    first launch), further calls leave the device's free memory unchanged.
    Starting from centers held in host memory gives fcm_run's result."""
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
    V0 = np.array([5.0, 45.0, 100.0, 160.0], dtype=np.float32)

    h = ctypes.c_void_p()
    assert L.fcm_create(ctypes.byref(h), 0, None) == 0
    try:
        Uref = torch.empty_like(U0)
        Vref = V0.copy()
        rep_ref = _lib.fcm_report()
        assert L.fcm_run(h, _p(xd), n, C, 2.0, 1e-5, 300, _lib.FCM_INIT_V, None, _p(Uref),
                         ctypes.c_void_p(Vref.ctypes.data), 0, ctypes.byref(rep_ref)) == _lib.FCM_OK
    finally:
        L.fcm_destroy(h)
    Uref = Uref.cpu().numpy()

    U = torch.empty_like(U0)
    Vd = torch.empty(C, dtype=torch.float32, device=dev)

    def call_u():
        return L.fcm_run_noalloc(_p(xd), n, C, 2.0, 1e-5, 300, _lib.FCM_INIT_U, _p(U0), _p(U), _p(Vd),
                                 None, None)

    def call_v(Vh):
        rep = _lib.fcm_report()
        st = L.fcm_run_noalloc(_p(xd), n, C, 2.0, 1e-5, 300, _lib.FCM_INIT_V, None, _p(U),
                               ctypes.c_void_p(Vh.ctypes.data), None, ctypes.byref(rep))
        return st, rep

    assert call_u() == _lib.FCM_OK
    assert call_v(V0.copy())[0] == _lib.FCM_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    assert call_u() == _lib.FCM_OK
    Vh = V0.copy()
    st, rep = call_v(Vh)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0, (free0, free1)
    assert st == _lib.FCM_OK and rep.iters == rep_ref.iters
    assert np.max(np.abs(U.cpu().numpy() - Uref)) <= U_TOL
    assert center_err(Vh, Vref) <= 1e-5


def test_noalloc_refuses_a_capturing_stream():
    import torch

    from paper_1601_00072_gb300 import _build, _lib
    _build.build()
    L = _lib.load()
    x, _, u0, C = phantom.single_image("phantom200")
    dev = torch.device("cuda", 0)
    xd = torch.from_numpy(x.astype(np.float32)).to(dev)
    U0 = torch.from_numpy(u0).to(dev)
    U = torch.empty_like(U0)
    V = torch.empty(C, dtype=torch.float32, device=dev)
    # the first call on the device comes before any capture
    assert L.fcm_run_noalloc(_p(xd), x.size, C, 2.0, 1e-5, 300, _lib.FCM_INIT_U, _p(U0), _p(U), _p(V),
                             None, None) == _lib.FCM_OK
    s = torch.cuda.Stream(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            V.mul_(1.0)  # the captured graph is not empty
            st = L.fcm_run_noalloc(_p(xd), x.size, C, 2.0, 1e-5, 300, _lib.FCM_INIT_U, _p(U0), _p(U), _p(V),
                                   ctypes.c_void_p(s.cuda_stream), None)
        finally:
            g.capture_end()
    assert st == _lib.FCM_ERR_INVALID_ARG
