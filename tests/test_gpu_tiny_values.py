"""Parity with the FP64 oracle on images whose intensities are tiny (needs a GPU).

The C ABI takes any finite float, not only grey levels. Two scales probe the
bottom of the FP32 range:

* intensities scaled by 2^-70 (about 1e-21 per grey level): every squared
  distance (x - v)^2 is below the smallest normal float, although the
  distances themselves are normal numbers;
* intensities scaled by 2^-15 (at most 7.8e-3) with C = 8: the products of
  seven squared distances that the m = 2 product form of Eq. 4 builds fall
  below the smallest normal float.

Eq. 4 depends only on ratios of distances, so on either scale the memberships
and iteration counts equal those of the unscaled image and the centers scale
with it (scaling by a power of two is exact). The oracle runs in FP64 on the
same scaled values, where none of these quantities underflows.
"""
import numpy as np
import pytest

import oracle
import phantom
from parity import assert_within, eps32, precision_report

pytestmark = pytest.mark.gpu

EPS = 1e-5
MAX_ITER = 300
EIGHT_MEANS = (0.0, 30.0, 60.0, 95.0, 130.0, 165.0, 200.0, 235.0)


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


def _gpu(fcm, x, C, m, u0, max_iter, path):
    from paper_1601_00072_gb300.fcm import Slice
    if path == "batched":
        s = Slice(x=_cuda(x), C=C, m=m, eps=EPS, max_iter=max_iter, U0=_cuda(u0))
        fcm.run_batched([s], tune=False)
        return s.iters, s.U.cpu().numpy(), s.V.cpu().numpy()
    kw = {"persistent": False} if path == "pass" else {"recompute": True} if path == "recompute" else {}
    r = fcm.run(_cuda(x), C, m, EPS, max_iter, U=_cuda(u0), **kw)
    return r.iters, r.U.cpu().numpy(), r.V.cpu().numpy()


def _check(fcm, x, C, m, u0, scale, path):
    """Both sides on the same scaled input, compared at the same iterate; the
    centers are compared after dividing by the scale."""
    xs = x.astype(np.float64) * scale
    assert np.array_equal(xs.astype(np.float32).astype(np.float64), xs)  # exact in FP32
    gi, gU, gV = _gpu(fcm, xs, C, m, u0, MAX_ITER, path)
    o = oracle.fcm(xs, C, m, eps32(EPS), MAX_ITER, U0=u0)
    d_iters = gi - o["iters"]
    k = min(gi, o["iters"])
    if gi > k:
        gi, gU, gV = _gpu(fcm, xs, C, m, u0, k, path)
    if o["iters"] > k:
        o = oracle.fcm(xs, C, m, eps32(EPS), k, U0=u0)
    assert np.all(np.isfinite(gU)) and np.all(np.isfinite(gV))
    rep = precision_report(gU, gV.astype(np.float64) / scale, gi + d_iters, o["U"], o["V"] / scale, o["iters"])
    assert_within(rep)
    return rep


@pytest.mark.parametrize("path", ["run", "pass", "recompute", "batched"])
@pytest.mark.parametrize("m", [2.0, 3.0, 2.5])
def test_squared_distances_below_the_normal_range(fcm, m, path):
    x, _, u0, C = phantom.single_image("phantom200")
    _check(fcm, x, C, m, u0, 2.0 ** -70, path)


@pytest.mark.parametrize("path", ["run", "pass", "recompute", "batched"])
@pytest.mark.parametrize("m", [2.0, 3.0])
def test_eight_clusters_on_small_intensities(fcm, m, path):
    img, _ = phantom.phantom2d(17, 160, 160, 4.0, EIGHT_MEANS)
    x = img.reshape(-1)
    u0 = phantom.dirichlet_u0((17, 8), 8, x.size)
    _check(fcm, x, 8, m, u0, 2.0 ** -15, path)
