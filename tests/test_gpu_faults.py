"""Failures made on the host, and what the library returns (needs a GPU).

Nothing here faults, traps or hangs the GPU:

* A grid-wide barrier is made to run out by asking it to wait for one arrival
  beyond the grid's own, which nothing ever makes (``barrier_phantoms``), with
  a short poll limit. Every block gives up at the first barrier, records
  FCM_ERR_TIMEOUT and returns; the same handle then runs the image correctly.
* An allocation is made to fail by the library's own allocation wrapper
  (``fail_alloc_in``) before it calls cudaMalloc at all; the entry point
  returns FCM_ERR_OOM and a later call completes the workspace.
"""
import numpy as np
import pytest

import phantom

pytestmark = pytest.mark.gpu

SHORT_SPINS = 2000  # about 0.3 ms of polling per barrier


@pytest.fixture(scope="module")
def lib():
    from paper_1601_00072_gb300 import _build, _lib
    _build.build()
    return _lib


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _image():
    x, _, u0, C = phantom.single_image("phantom200")
    return x, u0, C


def _run(h, x, u0, C, **kw):
    r = h.run(_cuda(x), C, 2.0, 1e-5, 300, U=_cuda(u0), raise_on_error=False, **kw)
    return r.status, r.iters, r.U.cpu().numpy(), r.V.cpu().numpy()


@pytest.mark.parametrize("kw", [{}, {"recompute": True}], ids=["whole_run", "u_free"])
def test_grid_barrier_gives_up_and_the_handle_recovers(lib, kw):
    from paper_1601_00072_gb300.fcm import FCM
    x, u0, C = _image()
    with FCM(0) as ref_h:
        ref = _run(ref_h, x, u0, C, **kw)
    assert ref[0] == lib.FCM_OK
    with FCM(0) as h:
        h.set_limits(grid_wait_spins=SHORT_SPINS, barrier_phantoms=1)
        assert h.limits()["barrier_phantoms"] == 1
        st, iters, _, _ = _run(h, x, u0, C, **kw)
        assert st == lib.FCM_ERR_TIMEOUT and iters == 0
        # the same handle, limits back to the defaults: the normal result, bit for bit
        h.set_limits(defaults=True)
        st, iters, U, V = _run(h, x, u0, C, **kw)
        assert st == ref[0] and iters == ref[1]
        assert np.array_equal(U, ref[2]) and np.array_equal(V, ref[3])


def test_multi_feature_barrier_gives_up(lib):
    from paper_1601_00072_gb300.fcm import FCM
    xm, _ = phantom.multichannel2d(5, 128, 128, 8.0, [(0.0, 40.0, 110.0, 150.0), (0.0, 150.0, 90.0, 60.0)])
    u0 = phantom.dirichlet_u0((5, 2), 4, xm.shape[1])
    with FCM(0) as h:
        ref = h.run_multi(_cuda(xm), 4, 2.0, 1e-5, 300, U0=_cuda(u0))
        h.set_limits(grid_wait_spins=SHORT_SPINS, barrier_phantoms=1)
        r = h.run_multi(_cuda(xm), 4, 2.0, 1e-5, 300, U0=_cuda(u0), raise_on_error=False)
        assert r.status == lib.FCM_ERR_TIMEOUT
        h.set_limits(defaults=True)
        r2 = h.run_multi(_cuda(xm), 4, 2.0, 1e-5, 300, U0=_cuda(u0))
        assert r2.iters == ref.iters and np.array_equal(r2.V.cpu().numpy(), ref.V.cpu().numpy())


@pytest.mark.parametrize("plan", [dict(schedule="rounds", block=512, tile=4096),
                                  dict(schedule="teams", block=256, tile=10)], ids=["rounds", "teams"])
def test_batch_barrier_gives_up(lib, plan):
    from paper_1601_00072_gb300.fcm import FCM, Slice

    def batch():
        out = []
        for i in range(6):
            sp, img, _ = phantom.batch_slice(i)
            x = img.reshape(-1)
            out.append(Slice(x=_cuda(x), C=sp.C, U0=_cuda(phantom.dirichlet_u0((phantom.U0_FAMILY, i), sp.C, x.size))))
        return out

    with FCM(0) as h:
        h.set_batched_plan(**plan)
        ref = batch()
        h.run_batched(ref)
        h.set_limits(grid_wait_spins=SHORT_SPINS, barrier_phantoms=1)
        bad = batch()
        st = h.run_batched(bad)
        assert st == lib.FCM_ERR_TIMEOUT
        if plan["schedule"] == "rounds":
            assert all(s.status == lib.FCM_ERR_TIMEOUT for s in bad)
        else:  # a slice of a lone CTA has no barrier; every team's gives up
            assert any(s.status == lib.FCM_ERR_TIMEOUT for s in bad)
            assert all(s.status in (lib.FCM_ERR_TIMEOUT, lib.FCM_OK) for s in bad)
        h.set_limits(defaults=True)
        again = batch()
        h.run_batched(again)
        for a, r in zip(again, ref):
            assert a.status == r.status and a.iters == r.iters
            assert np.array_equal(a.V.cpu().numpy(), r.V.cpu().numpy())


@pytest.mark.parametrize("nth", [1, 2, 3])
def test_injected_allocation_failure_returns_oom(lib, nth):
    from paper_1601_00072_gb300.fcm import FCM
    x, u0, C = _image()
    with FCM(0) as ref_h:
        ref = _run(ref_h, x, u0, C)
    with FCM(0) as h:
        h.set_limits(fail_alloc_in=nth)
        st, _, _, _ = _run(h, x, u0, C)
        assert st == lib.FCM_ERR_OOM
        assert h.limits()["fail_alloc_in"] == 0  # the injection fired once
        st, iters, U, V = _run(h, x, u0, C)
        assert st == ref[0] and iters == ref[1] and np.array_equal(V, ref[3])


def test_injected_allocation_failure_in_a_batch(lib):
    from paper_1601_00072_gb300 import _lib
    from paper_1601_00072_gb300.fcm import FCM, Slice
    sp, img, _ = phantom.batch_slice(3)
    x = img.reshape(-1)
    u0 = phantom.dirichlet_u0((phantom.U0_FAMILY, 3), sp.C, x.size)
    with FCM(0) as h:
        h.set_limits(fail_alloc_in=4)
        with pytest.raises(_lib.FcmError) as e:
            h.run_batched([Slice(x=_cuda(x), C=sp.C, U0=_cuda(u0))], tune=False)
        assert e.value.status == lib.FCM_ERR_OOM
        s = Slice(x=_cuda(x), C=sp.C, U0=_cuda(u0))
        assert h.run_batched([s], tune=False) in (lib.FCM_OK, lib.FCM_NOT_CONVERGED)
        assert s.status == lib.FCM_OK and s.iters > 1
