"""Parity of the batched histogram-domain path (fcm_run_batched_hist) with the
FP64 oracle (needs a GPU).

The same uneven 8-bit slices as the batched per-pixel tests, run one CTA per
slice on their 256-bin histograms. Each slice is compared with the oracle's
k-th iterate at the CUDA run's own k, the iteration counts within one, with
the same handling of trajectory-sensitive slices.
"""
import numpy as np
import pytest

import oracle
import phantom
from parity import assert_within, eps32, precision_report
from test_gpu_batched import _cuda, assert_batch, assert_slice, check_slice, make_batch

pytestmark = pytest.mark.gpu

EPS = 1e-5


@pytest.fixture(scope="module")
def fcm():
    from paper_1601_00072_gb300 import _build
    _build.build()
    from paper_1601_00072_gb300.fcm import FCM
    h = FCM(0)
    yield h
    h.close()


def test_batch_from_memberships(fcm):
    slices, host = make_batch(range(48))
    st = fcm.run_batched_hist(slices)
    assert st in (0, 1)
    assert_batch(slices, host)


def test_batch_from_centers(fcm):
    slices, host = make_batch(range(48, 80), init="V")
    assert fcm.run_batched_hist(slices) in (0, 1)
    assert_batch(slices, host)


@pytest.mark.parametrize("m", [1.5, 3.0, 2.5])
def test_other_fuzzifiers(fcm, m):
    slices, host = make_batch(range(100, 116), m=m)
    assert fcm.run_batched_hist(slices) in (0, 1)
    assert_batch(slices, host, m)


def test_full_512_slice_batch(fcm):
    slices, host = make_batch(range(512))
    assert fcm.run_batched_hist(slices) in (0, 1)
    sensitive = 0
    for i, (s, (x, u0, V0)) in enumerate(zip(slices, host)):
        rep, _ = check_slice(s, x, u0, V0, 2.0)
        assert s.status in (0, 1), (i, s.status)
        assert_slice(rep, f"slice {i} (n={s.x.numel()}, C={s.C})")
        sensitive += rep["conditioning"] == "sensitive"
    assert sensitive <= 3  # of the 13 slices the oracle marks trajectory-sensitive


def test_ragged_and_tiny_slices(fcm):
    """Sizes from one pixel up, odd sizes, and C up to 8."""
    from paper_1601_00072_gb300.fcm import Slice
    img, _ = phantom.phantom2d(71, 64, 64, 9.0)
    flat = img.reshape(-1)
    cases = [(1, 1), (3, 2), (17, 3), (255, 4), (1001, 5), (4095, 8), (4096, 6)]
    slices, host = [], []
    for t, (n, C) in enumerate(cases):
        x = flat[:n].copy()
        u0 = phantom.dirichlet_u0((71, t), C, n)
        slices.append(Slice(x=_cuda(x), C=C, eps=EPS, max_iter=300, U0=_cuda(u0)))
        host.append((x, u0))
    assert fcm.run_batched_hist(slices) in (0, 1)
    for (x, u0), s in zip(host, slices):
        o = oracle.fcm_quantized(x, s.C, 2.0, eps32(EPS), 300, U0=u0)
        assert abs(s.iters - o["iters"]) <= 1, (x.size, s.C, s.iters, o["iters"])
        at = oracle.fcm_quantized(x, s.C, 2.0, 0.0, s.iters, U0=u0)
        ref_U = oracle.memberships(np.arange(256.0), at["V"], 2.0)[:, x]
        rep = precision_report(s.U.cpu().numpy(), s.V.cpu().numpy(), s.iters, ref_U, at["V"], s.iters)
        assert_within(rep)


def test_non_grey_level_slice_is_rejected_alone(fcm):
    """A slice holding a non-integer intensity gets FCM_ERR_BAD_INPUT, its U
    is left as it was and V = V^0 (0 from a U^0); the other slices run."""
    import torch
    from paper_1601_00072_gb300 import _lib
    slices, host = make_batch(range(200, 204))
    bad = slices[1]
    xb = bad.x.clone()
    xb[7] = 12.5
    bad.x = xb
    bad.U = torch.full((bad.C, xb.numel()), -1.0, device=xb.device)
    st = fcm.run_batched_hist(slices)
    assert st == _lib.FCM_ERR_BAD_INPUT
    assert bad.status == _lib.FCM_ERR_BAD_INPUT and bad.iters == 0
    assert bool((bad.U == -1.0).all())
    assert np.array_equal(bad.V.cpu().numpy(), np.zeros(bad.C, np.float32))
    for i in (0, 2, 3):
        rep, _ = check_slice(slices[i], *host[i], 2.0)
        assert slices[i].status in (0, 1)
        assert_slice(rep, f"slice {i}")


def test_exact_first_stop_where_the_bound_cannot_decide(fcm):
    """The first stopping quantity delta_1 = max_i |f(x_i, V^1) - U^0_i| is
    bounded from below by one pixel per grey level; a pass over every pixel
    takes it exactly only when that bound is below eps or max_iter is 1.
    Slices whose U^0 already sits at a fixed point (the oracle's converged
    memberships) stop at iteration 1 with delta_1 of order 1e-7; a slice with
    max_iter = 1 stops there too; the others, in the same batch, need no
    exact pass. Each is compared with the oracle at the same iterate."""
    from paper_1601_00072_gb300.fcm import Slice
    slices, host = [], []
    for t, i in enumerate(range(300, 306)):
        sp, img, _ = phantom.batch_slice(i)
        x = img.reshape(-1)
        u0 = phantom.dirichlet_u0((phantom.U0_FAMILY, i), sp.C, x.size)
        max_iter = 300
        if t in (0, 3):
            o = oracle.fcm_quantized(x, sp.C, 2.0, 1e-10, 2000, U0=u0, want_U=False)
            u0 = np.ascontiguousarray(oracle.memberships(np.arange(256.0), o["V"], 2.0)[:, x], dtype=np.float32)
        if t == 1:
            max_iter = 1
        slices.append(Slice(x=_cuda(x), C=sp.C, eps=EPS, max_iter=max_iter, U0=_cuda(u0)))
        host.append((x, u0, max_iter))
    assert fcm.run_batched_hist(slices) in (0, 1)
    for t, (s, (x, u0, mi)) in enumerate(zip(slices, host)):
        o = oracle.fcm_quantized(x, s.C, 2.0, eps32(EPS), mi, U0=u0)
        if t in (0, 3):
            assert s.status == 0 and s.iters == 1 and o["iters"] == 1, (t, s.iters, o["iters"])
        if t == 1:
            assert s.status == 1 and s.iters == 1
        if t in (0, 1, 3):
            # delta_1 itself, over every pixel
            assert abs(s.delta - o["delta"][0]) <= 1e-6, (t, s.delta, o["delta"][0])
        assert abs(s.iters - o["iters"]) <= 1, (t, s.iters, o["iters"])
        at = oracle.fcm_quantized(x, s.C, 2.0, 0.0, s.iters, U0=u0)
        ref_U = oracle.memberships(np.arange(256.0), at["V"], 2.0)[:, x]
        rep = precision_report(s.U.cpu().numpy(), s.V.cpu().numpy(), s.iters, ref_U, at["V"], s.iters)
        if t == 1:
            # V^1 from a random U^0 puts every center near the mean grey level,
            # where U^1 = f(x, V^1) magnifies the rounding of V^1 (as in the
            # early iterates of the single-image runs): V^1 and delta_1 only
            assert rep["center_rel_err"] <= 1e-5, rep
        else:
            assert_within(rep)
