"""Reductions of known sequences, and canaries around the output buffers
(needs a GPU).

Reductions: with C = 1 every membership is exactly 1 (Eq. 4), so V^1 is the
mean of x (Eq. 3) and the run stops after iteration 1 (U^1 = U^0 = 1). For
integer-valued x the FP32 partial sums of a thread, a warp and a block stay
exact (below 2^24), and the cross-block sums are double-float, so the
center must equal the FP64 mean to the accuracy of the double-float
quotient, at every size: one pixel, ragged tails that take the plain-load
kernel, and 10^7 pixels.

Canaries: compute-sanitizer is closed on this machine, so every path writes U
and V into the middle of larger buffers filled with a sentinel, and the
sentinel must come back untouched.
"""
import numpy as np
import pytest

import phantom

pytestmark = pytest.mark.gpu

SENTINEL = np.float32(-12345.678)
PAD = 1024  # floats on each side; a multiple of 4 keeps the 16-byte alignment


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


def _sequence(kind, n):
    return np.ones(n, np.float32) if kind == "ones" else (np.arange(n) % 256).astype(np.float32)


@pytest.mark.parametrize("kind", ["ones", "ramp"])
@pytest.mark.parametrize("n", [1, 7, 4099, 1 << 20, 10_000_000, 10_000_003])
def test_center_is_the_exact_mean(fcm, kind, n):
    x = _sequence(kind, n)
    r = fcm.run(_cuda(x), 1, 2.0, 1e-5, 300, U0=_cuda(np.ones((1, n), np.float32)))
    mean = float(np.sum(x, dtype=np.float64)) / n  # exact: integers below 2^53
    assert r.status == 0 and r.iters == 1
    assert abs(r.V64[0] - mean) <= 1e-12 * max(mean, 1.0), (r.V64[0], mean)
    assert abs(float(r.V.cpu().numpy()[0]) - mean) <= 6e-8 * max(mean, 1.0)
    J = float(np.sum((x.astype(np.float64) - mean) ** 2))
    assert abs(r.J - J) <= 1e-5 * max(J, 1.0), (r.J, J)  # FP32 per-thread sums of (x - v)^2


@pytest.mark.parametrize("path", [{"recompute": True}, {"persistent": False}, {"tma": False},
                                  {"deterministic": True}])
def test_center_is_the_exact_mean_on_every_path(fcm, path):
    n = 10_000_000
    x = _sequence("ramp", n)
    r = fcm.run(_cuda(x), 1, 2.0, 1e-5, 300, U0=_cuda(np.ones((1, n), np.float32)), **path)
    mean = float(np.sum(x, dtype=np.float64)) / n
    assert r.status == 0 and r.iters == 1
    assert abs(r.V64[0] - mean) <= 1e-12 * mean, (path, r.V64[0], mean)


def _padded(C, n, host=False):
    """A buffer of PAD + C*n + PAD floats filled with the sentinel, and the
    [C, n] view of its middle (16-byte aligned)."""
    import torch
    buf = torch.full((2 * PAD + C * n,), float(SENTINEL), dtype=torch.float32,
                     device="cpu" if host else "cuda")
    if host:
        buf = buf.pin_memory()
    return buf, buf[PAD:PAD + C * n].view(C, n)


def _untouched(buf, C, n):
    b = buf.cpu().numpy()
    return bool(np.all(b[:PAD] == SENTINEL) and np.all(b[PAD + C * n:] == SENTINEL))


@pytest.mark.parametrize("kw", [{}, {"persistent": False}, {"tma": False}, {"recompute": True}])
@pytest.mark.parametrize("side", [200, 203])
def test_single_image_writes_stay_inside_U_and_V(fcm, kw, side):
    if kw.get("recompute") and (side * side) % 4:
        pytest.skip("the U-free run needs n % 4 == 0")
    img, _ = phantom.phantom2d(41, side, side, 8.0)
    x = img.reshape(-1)
    n, C = x.size, 4
    u0 = phantom.dirichlet_u0((41, side), C, n)
    ub, U = _padded(C, n)
    vb, V = _padded(1, C)
    r = fcm.run(_cuda(x), C, 2.0, 1e-5, 300, U0=_cuda(u0), U=U, V=V.view(C), **kw)
    assert r.status == 0
    assert _untouched(ub, C, n) and _untouched(vb, 1, C)


def test_histogram_and_stream_writes_stay_inside_U_and_V(fcm):
    img, _ = phantom.phantom2d(42, 256, 256, 8.0)
    x = img.reshape(-1)
    n, C = x.size, 4
    u0 = phantom.dirichlet_u0((42, 1), C, n)
    ub, U = _padded(C, n)
    vb, V = _padded(1, C)
    r = fcm.run_hist(_cuda(x), C, 2.0, 1e-5, 300, U0=_cuda(u0), U=U, V=V.view(C))
    assert r.status == 0 and _untouched(ub, C, n) and _untouched(vb, 1, C)
    # host-resident sequence: every image's U lands in its own padded pinned buffer
    import torch
    xs = [torch.from_numpy(x.astype(np.float32)).pin_memory() for _ in range(3)]
    u0s = [torch.from_numpy(u0).pin_memory() for _ in range(3)]
    bufs = [_padded(C, n, host=True) for _ in range(3)]
    res = fcm.run_stream(xs, C, 2.0, 1e-5, 300, U0s=u0s, Us=[u for _, u in bufs])
    assert all(q.status == 0 for q in res)
    assert all(_untouched(b, C, n) for b, _ in bufs)


@pytest.mark.parametrize("kind", ["pixels", "histogram"])
def test_batched_writes_stay_inside_U_and_V(fcm, kind):
    from paper_1601_00072_gb300.fcm import Slice
    sl, bufs = [], []
    for i, (hh, ww, C) in enumerate(((64, 80, 3), (131, 97, 4), (256, 256, 5), (1, 1, 2))):
        im, _ = phantom.phantom2d(50 + i, hh, ww, 6.0)
        x = im.reshape(-1)
        n = x.size
        ub, U = _padded(C, n)
        vb, V = _padded(1, C)
        sl.append(Slice(x=_cuda(x), C=C, U0=_cuda(phantom.dirichlet_u0((50 + i, 1), C, n)), U=U, V=V.view(C)))
        bufs.append((ub, vb, C, n))
    st = fcm.run_batched(sl) if kind == "pixels" else fcm.run_batched_hist(sl)
    assert st in (0, 1)
    for ub, vb, C, n in bufs:
        assert _untouched(ub, C, n) and _untouched(vb, 1, C)
