"""Parity of the multi-feature CUDA run (fcm_run_multi) with the FP64
multi-feature oracle (needs a GPU).

Inputs are multi-channel phantoms: one seeded label layout rendered with a
different class-mean table per channel (like co-registered MR sequences with
different tissue contrasts), each channel with its own noise.
"""
import numpy as np
import pytest

import oracle
import phantom
from parity import eps32

pytestmark = pytest.mark.gpu

EPS = 1e-5
MAX_ITER = 300
CONTRASTS = [(0.0, 40.0, 110.0, 150.0), (0.0, 150.0, 90.0, 60.0), (10.0, 200.0, 120.0, 80.0),
             (0.0, 30.0, 30.0, 160.0)]


@pytest.fixture(scope="module")
def fcm():
    from paper_1601_00072_gb300 import _build
    _build.build()
    from paper_1601_00072_gb300.fcm import FCM
    h = FCM(0)
    yield h
    h.close()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


# eight tissue classes per channel, for runs with eight clusters
CONTRASTS8 = [tuple(float(v) for v in np.linspace(0, 245, 8)),
              tuple(float(v) for v in np.linspace(240, 10, 8)),
              (0.0, 200.0, 60.0, 160.0, 30.0, 230.0, 100.0, 130.0),
              (50.0, 10.0, 90.0, 240.0, 130.0, 170.0, 210.0, 20.0)]


def multi_phantom(seed, H, W, D, sigma=8.0, classes=4):
    return phantom.multichannel2d(seed, H, W, sigma, (CONTRASTS if classes == 4 else CONTRASTS8)[:D])


def gpu(fcm, x, C, m, max_iter=MAX_ITER, u0=None, V0=None):
    if u0 is not None:
        r = fcm.run_multi(_cuda(x), C, m, EPS, max_iter, U0=_cuda(u0))
    else:
        r = fcm.run_multi(_cuda(x), C, m, EPS, max_iter, V0=_cuda(V0))
    return r, r.U.cpu().numpy(), r.V.cpu().numpy()


def orc(x, C, m, max_iter=MAX_ITER, u0=None, V0=None):
    return oracle.fcm_multi(x.astype(np.float64), C, m, eps32(EPS), max_iter, U0=u0, V0=V0)


def check(fcm, x, C, m, u0=None, V0=None):
    g, gU, gV = gpu(fcm, x, C, m, u0=u0, V0=V0)
    o = orc(x, C, m, u0=u0, V0=V0)
    assert abs(g.iters - o["iters"]) <= 1, (g.iters, o["iters"])
    k = min(g.iters, o["iters"])
    if g.iters > k:
        g, gU, gV = gpu(fcm, x, C, m, max_iter=k, u0=u0, V0=V0)
    if o["iters"] > k:
        o = orc(x, C, m, max_iter=k, u0=u0, V0=V0)
    cerr = np.max(np.abs(gV - o["V"]) / np.maximum(np.abs(o["V"]), 1.0))
    uerr = np.max(np.abs(gU - o["U"]))
    agree = np.mean(np.argmax(gU, 0) == np.argmax(o["U"], 0))
    assert cerr <= 1e-5 and uerr <= 1e-5 and agree >= 0.9999, (cerr, uerr, agree)
    assert abs(g.J - o["J"][-1]) <= 1e-5 * abs(o["J"][-1])
    return g


@pytest.mark.parametrize("D", [1, 2, 3, 4])
@pytest.mark.parametrize("m", [2.0, 2.5])
def test_phantom_channels_match_oracle(fcm, D, m):
    x, _ = multi_phantom(21, 120, 110, D)
    u0 = phantom.dirichlet_u0((21, D), 4, x.shape[1])
    check(fcm, x, 4, m, u0=u0)


@pytest.mark.parametrize("n,D,C", [(1, 2, 1), (7, 3, 2), (4099, 2, 5), (30001, 4, 8), (65536, 3, 3)])
def test_ragged_sizes_and_cluster_counts(fcm, n, D, C):
    side = int(np.ceil(np.sqrt(n)))
    x, _ = multi_phantom(300 + n, side, side, D, classes=8 if C > 4 else 4)
    x = np.ascontiguousarray(x[:, :n])
    u0 = phantom.dirichlet_u0((300 + n, 2), C, n)
    check(fcm, x, C, 2.0, u0=u0)


def test_init_from_centers(fcm):
    x, _ = multi_phantom(22, 100, 100, 2)
    V0 = np.array([[5.0, 5.0], [45.0, 140.0], [100.0, 95.0], [145.0, 65.0]])
    g = check(fcm, x, 4, 2.0, V0=V0)
    assert g.V64.shape == (4, 2)


def test_one_channel_matches_the_scalar_cuda_run(fcm):
    x, _, u0, C = phantom.single_image("phantom200")
    g, gU, gV = gpu(fcm, x[None, :].astype(np.float32), C, 2.0, u0=u0)
    s = fcm.run(_cuda(x), C, 2.0, EPS, MAX_ITER, U0=_cuda(u0))
    assert abs(g.iters - s.iters) <= 1
    sV = s.V.cpu().numpy()
    assert np.max(np.abs(gV[:, 0] - sV) / np.maximum(np.abs(sV), 1.0)) <= 1e-5


def test_non_finite_channel_value_is_rejected(fcm):
    x, _ = multi_phantom(23, 50, 50, 3)
    x = x.astype(np.float32)
    x[2, 77] = np.nan
    u0 = phantom.dirichlet_u0((23, 1), 3, x.shape[1])
    r = fcm.run_multi(_cuda(x), 3, 2.0, EPS, MAX_ITER, U0=_cuda(u0), raise_on_error=False)
    assert r.status == -4


def test_repeatable(fcm):
    x, _ = multi_phantom(24, 200, 200, 3)
    u0 = phantom.dirichlet_u0((24, 1), 4, x.shape[1])
    a = gpu(fcm, x, 4, 2.0, u0=u0)
    b = gpu(fcm, x, 4, 2.0, u0=u0)
    assert a[0].iters == b[0].iters and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
