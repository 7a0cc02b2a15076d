"""A sequence of images from host memory through fcm_run_stream (needs a GPU).

Each image of the sequence must come out exactly as a single fcm_run of the
same image on the device (same whole-run kernel, same inputs), and within the
parity bar of the FP64 oracle at the same iterate. Five images exercise the
reuse of the three staging sets (images i and i + 3 share one).
"""
import numpy as np
import pytest

import oracle
import phantom
from parity import assert_within, eps32, precision_report

pytestmark = pytest.mark.gpu

EPS = 1e-5
MAX_ITER = 300
C = 4
SIDE = 200  # n = 40,000, a multiple of 4


@pytest.fixture(scope="module")
def fcm():
    from paper_1601_00072_gb300 import _build
    _build.build()
    from paper_1601_00072_gb300.fcm import FCM
    h = FCM(0)
    yield h
    h.close()


def images(k, first=501):
    out = []
    for s in range(first, first + k):
        img, _ = phantom.phantom2d(s, SIDE, SIDE, 6.0 + (s % 5))
        x = img.reshape(-1).astype(np.float32)
        u0 = phantom.dirichlet_u0((s, 3), C, x.size)
        out.append((x, u0))
    return out


def pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()


def single(fcm, x, u0, m, max_iter=MAX_ITER, recompute=False):
    import torch
    r = fcm.run(torch.from_numpy(x).cuda(), C, m, EPS, max_iter, U=torch.from_numpy(u0).cuda(),
                recompute=recompute)
    return r, r.U.cpu().numpy(), r.V.cpu().numpy()


def oracle_at(x, u0, m, iters):
    """The oracle's own run, and its iterate at the CUDA run's count."""
    o = oracle.fcm(x.astype(np.float64), C, m, eps32(EPS), MAX_ITER, U0=u0)
    at = o if o["iters"] == iters else oracle.fcm(x.astype(np.float64), C, m, 0.0, iters, U0=u0)
    return o, at


@pytest.mark.parametrize("m", [2.0, 3.0])
def test_stream_equals_single_runs_and_oracle(fcm, m):
    imgs = images(5)
    res = fcm.run_stream([pinned(x) for x, _ in imgs], C, m, EPS, MAX_ITER,
                         U0s=[pinned(u) for _, u in imgs])
    assert len(res) == 5
    for i, ((x, u0), r) in enumerate(zip(imgs, res)):
        s, sU, sV = single(fcm, x, u0, m)
        assert r.status == s.status and r.iters == s.iters, (i, r.iters, s.iters)
        assert np.array_equal(r.U.numpy(), sU), i
        assert np.array_equal(np.asarray(r.V), sV), i
        assert np.array_equal(r.V64, s.V64) and r.J == s.J, i
        o, at = oracle_at(x, u0, m, r.iters)
        assert abs(r.iters - o["iters"]) <= 1, (i, r.iters, o["iters"])
        rep = precision_report(r.U.numpy(), np.asarray(r.V), r.iters, at["U"], at["V"], r.iters,
                               r.J, at["J"][-1])
        assert_within(rep)


def test_u0_in_place_and_pageable_numpy(fcm):
    """U0 read from the output buffers themselves; plain numpy inputs."""
    imgs = images(3, first=601)
    Us = [np.ascontiguousarray(u0, dtype=np.float32).copy() for _, u0 in imgs]
    res = fcm.run_stream([x for x, _ in imgs], C, 2.0, EPS, MAX_ITER, Us=Us)
    for (x, u0), r, Ui in zip(imgs, res, Us):
        s, sU, sV = single(fcm, x, u0, 2.0)
        assert r.U is Ui
        assert r.iters == s.iters and np.array_equal(Ui, sU) and np.array_equal(np.asarray(r.V), sV)


def test_recompute_option(fcm):
    imgs = images(3, first=701)
    res = fcm.run_stream([pinned(x) for x, _ in imgs], C, 2.0, EPS, MAX_ITER,
                         U0s=[pinned(u) for _, u in imgs], recompute=True)
    for (x, u0), r in zip(imgs, res):
        s, sU, sV = single(fcm, x, u0, 2.0, recompute=True)
        assert r.iters == s.iters and np.array_equal(r.U.numpy(), sU)
        assert np.array_equal(np.asarray(r.V), sV)


def test_max_iter_reached_and_single_image(fcm):
    from paper_1601_00072_gb300 import _lib
    (x, u0), = images(1, first=801)
    res = fcm.run_stream([pinned(x)], C, 2.0, EPS, 4, U0s=[pinned(u0)])
    assert res[0].status == _lib.FCM_NOT_CONVERGED and res[0].iters == 4
    s, sU, sV = single(fcm, x, u0, 2.0, max_iter=4)
    assert np.array_equal(res[0].U.numpy(), sU) and np.array_equal(np.asarray(res[0].V), sV)
    o, at = oracle_at(x, u0, 2.0, 4)
    rep = precision_report(res[0].U.numpy(), np.asarray(res[0].V), 4, at["U"], at["V"], 4)
    assert_within(rep)


def test_rejects_unaligned_size(fcm):
    from paper_1601_00072_gb300 import _lib
    x = np.zeros(1001, np.float32)
    u = np.full((C, 1001), 0.25, np.float32)
    with pytest.raises(_lib.FcmError) as e:
        fcm.run_stream([x], C, 2.0, EPS, MAX_ITER, U0s=[u])
    assert e.value.status == _lib.FCM_ERR_INVALID_ARG
