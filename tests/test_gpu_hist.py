"""Parity of the histogram-domain CUDA path (fcm_run_hist) with the FP64
oracle (needs a GPU).

The oracle's 256-bin form takes Algorithm 1's steps on the grey-level
histogram and is pinned to the per-pixel oracle (tests/oracle_pins.py), so
both definitions bind this path. Comparisons follow the single-image tests:
the CUDA run against the oracle's iterate at the CUDA run's own iteration
count, and the counts within one.
"""
import numpy as np
import pytest

import oracle
import phantom
from parity import assert_within, eps32, precision_report

pytestmark = pytest.mark.gpu

EPS = 1e-5
MAX_ITER = 300


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


def gpu_hist(fcm, x, C, m, eps=EPS, max_iter=MAX_ITER, u0=None, V0=None, raise_on_error=True):
    xt = _cuda(x)
    if u0 is not None:
        r = fcm.run_hist(xt, C, m, eps, max_iter, U0=_cuda(u0), raise_on_error=raise_on_error)
    else:
        r = fcm.run_hist(xt, C, m, eps, max_iter, V0=_cuda(V0), raise_on_error=raise_on_error)
    return r, r.U.cpu().numpy(), r.V.cpu().numpy()


def oracle_q(x, C, m, eps, max_iter, u0=None, V0=None, want_U=True):
    return oracle.fcm_quantized(np.asarray(x, np.uint8), C, m, eps32(eps), max_iter, U0=u0, V0=V0,
                                want_U=want_U)


def paired(fcm, x, C, m, u0=None, V0=None, sample=None):
    g, gU, gV = gpu_hist(fcm, x, C, m, u0=u0, V0=V0)
    o = oracle_q(x, C, m, EPS, MAX_ITER, u0=u0, V0=V0, want_U=sample is None)
    d_iters = g.iters - o["iters"]
    k = min(g.iters, o["iters"])
    if g.iters > k:
        g, gU, gV = gpu_hist(fcm, x, C, m, max_iter=k, u0=u0, V0=V0)
    if o["iters"] > k:
        o = oracle_q(x, C, m, EPS, k, u0=u0, V0=V0, want_U=sample is None)
    if sample is None:
        oU, gUs = o["U"], gU
    else:
        oU = oracle.memberships(np.arange(256.0), o["V"], m)[:, np.asarray(x)[sample]]
        gUs = gU[:, sample]
    rep = precision_report(gUs, gV, g.iters + d_iters, oU, o["V"], o["iters"], g.J, o["J"][-1])
    return rep, g, gU, gV, o


@pytest.mark.parametrize("m", [2.0, 1.5, 3.0, 2.5])
def test_phantom200_matches_oracle(fcm, m):
    x, _, u0, C = phantom.single_image("phantom200")
    rep, g, gU, *_ = paired(fcm, x, C, m, u0=u0)
    assert_within(rep)
    assert rep["J_rel_err"] < 1e-5
    assert np.max(np.abs(gU.sum(0) - 1.0)) < 1e-6
    assert g.launches == 5


def test_phantom1024_matches_oracle(fcm):
    x, _, u0, C = phantom.single_image("phantom1024")
    rep, *_ = paired(fcm, x, C, 2.0, u0=u0)
    assert_within(rep)


@pytest.mark.parametrize("m", [2.0, 3.0])
def test_volume256_matches_oracle(fcm, m):
    """The 16.7M-voxel volume; U compared on a 200k-voxel sample."""
    x, _, u0, C = phantom.single_image("volume256")
    idx = np.random.default_rng(0).choice(x.size, 200_000, replace=False)
    rep, *_ = paired(fcm, x, C, m, u0=u0, sample=idx)
    assert_within(rep)


def test_matches_the_per_pixel_cuda_path(fcm):
    """Same image, same U0: the histogram and per-pixel CUDA runs agree to the
    parity bars (they differ only in the order of rounding)."""
    x, _, u0, C = phantom.single_image("phantom200")
    g, gU, gV = gpu_hist(fcm, x, C, 2.0, u0=u0)
    p = fcm.run(_cuda(x), C, 2.0, EPS, MAX_ITER, U0=_cuda(u0))
    assert abs(p.iters - g.iters) <= 1
    pV = p.V.cpu().numpy()
    assert np.max(np.abs(pV - gV) / np.maximum(np.abs(pV), 1.0)) <= 1e-5


def test_init_from_centers_matches_oracle(fcm):
    x, _, _, C = phantom.single_image("phantom200")
    rep, g, *_ = paired(fcm, x, C, 2.0, V0=np.array([5.0, 45.0, 100.0, 160.0]))
    assert_within(rep)
    assert g.launches == 4


@pytest.mark.parametrize("n,C,m", [(1, 1, 2.0), (3, 2, 2.0), (1001, 3, 1.5), (4099, 5, 3.0),
                                   (65537, 8, 2.0), (123457, 4, 2.7), (40000, 1, 2.0), (777, 6, 2.0),
                                   (5000, 7, 1.5)])
def test_ragged_sizes_and_cluster_counts(fcm, n, C, m):
    side = int(np.ceil(np.sqrt(n)))
    img, _ = phantom.phantom2d(2000 + n, side, side, 9.0)
    x = img.reshape(-1)[:n]
    u0 = phantom.dirichlet_u0((2000 + n, 7), C, n)
    rep, *_ = paired(fcm, x, C, m, u0=u0)
    assert_within(rep)


def test_max_iter_reached(fcm):
    x, _, u0, C = phantom.single_image("phantom200")
    g, gU, gV = gpu_hist(fcm, x, C, 2.0, max_iter=30, u0=u0)
    assert g.status == 1 and g.iters == 30
    o = oracle_q(x, C, 2.0, EPS, 30, u0=u0)
    assert_within(precision_report(gU, gV, 30, o["U"], o["V"], o["iters"]))


@pytest.mark.parametrize("bad", ["fraction", "above", "negative", "nan"])
def test_non_grey_level_input_is_rejected(fcm, bad):
    x, _, u0, C = phantom.single_image("phantom200")
    x = x.astype(np.float32).copy()
    x[123] = {"fraction": 17.5, "above": 256.0, "negative": -1.0, "nan": np.nan}[bad]
    g, *_ = gpu_hist(fcm, x, C, 2.0, u0=u0, raise_on_error=False)
    assert g.status == -4


@pytest.mark.parametrize("bad", ["negative", "nan", "inf", "last"])
@pytest.mark.parametrize("m", [2.0, 2.5])
def test_invalid_u0_is_rejected(fcm, bad, m):
    """A negative entry is caught in the pixel pass; a NaN or infinite one
    through the non-finite V^1 sums it produces (m = 2.5 takes the generic
    power). The handle runs a good input correctly afterwards."""
    x, _, u0, C = phantom.single_image("phantom200")
    good = u0
    u0 = u0.copy()
    where = (C - 1, x.size - 1) if bad == "last" else (1, 5)
    u0[where] = {"negative": -0.25, "nan": np.nan, "inf": np.inf, "last": np.nan}[bad]
    g, *_ = gpu_hist(fcm, x, C, m, u0=u0, raise_on_error=False)
    assert g.status == -4
    g, gU, gV = gpu_hist(fcm, x, C, m, u0=good)
    o = oracle_q(x, C, m, EPS, MAX_ITER, u0=good)
    assert abs(g.iters - o["iters"]) <= 1 and g.status == 0


def test_repeatable(fcm):
    x, _, u0, C = phantom.single_image("phantom1024")
    a = gpu_hist(fcm, x, C, 2.0, u0=u0)
    b = gpu_hist(fcm, x, C, 2.0, u0=u0)
    assert a[0].iters == b[0].iters
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
