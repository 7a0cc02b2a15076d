"""Parity of the single-image CUDA path with the FP64 oracle (needs a GPU).

Every test calls the CUDA library through its C ABI (via the ctypes binding)
and compares with the oracle on the same seeded inputs.
"""
import numpy as np
import pytest

import oracle
import phantom
from parity import U_TOL, assert_within, center_err, eps32, precision_report

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


def gpu_run(fcm, x, C, m, eps=EPS, max_iter=MAX_ITER, u0=None, V0=None, **kw):
    xt = _cuda(x)
    if u0 is not None:
        r = fcm.run(xt, C, m, eps, max_iter, U=_cuda(u0), **kw)
    else:
        r = fcm.run(xt, C, m, eps, max_iter, V0=_cuda(V0), **kw)
    return r, r.U.cpu().numpy(), r.V.cpu().numpy()


def oracle_run(x, C, m, eps, max_iter, u0=None, V0=None, quantized=False, want_U=True):
    if quantized:
        return oracle.fcm_quantized(np.asarray(x, np.uint8), C, m, eps32(eps), max_iter,
                                    U0=u0, V0=V0, want_U=want_U)
    return oracle.fcm(np.asarray(x, np.float64), C, m, eps32(eps), max_iter, U0=u0, V0=V0,
                      want_U=want_U)


def paired(fcm, x, C, m, u0=None, V0=None, quantized=False, eps=EPS, max_iter=MAX_ITER):
    """Run both sides; if the iteration counts differ, rerun the longer one
    with max_iter equal to the shorter count, so both return the same iterate."""
    g, gU, gV = gpu_run(fcm, x, C, m, eps, max_iter, u0=u0, V0=V0)
    o = oracle_run(x, C, m, eps, max_iter, u0=u0, V0=V0, quantized=quantized)
    d_iters = g.iters - o["iters"]
    k = min(g.iters, o["iters"])
    if g.iters > k:
        g, gU, gV = gpu_run(fcm, x, C, m, eps, k, u0=u0, V0=V0)
    if o["iters"] > k:
        o = oracle_run(x, C, m, eps, k, u0=u0, V0=V0, quantized=quantized)
    rep = precision_report(gU, gV, g.iters + d_iters, o["U"], o["V"], o["iters"], g.J, o["J"][-1])
    return rep, g, gU, gV, o


@pytest.mark.parametrize("m", [2.0, 1.5, 3.0, 2.5])
def test_phantom200_matches_oracle(fcm, m):
    x, _, u0, C = phantom.single_image("phantom200")
    rep, g, gU, *_ = paired(fcm, x, C, m, u0=u0)
    assert_within(rep)
    assert rep["J_rel_err"] < 1e-5
    assert np.max(np.abs(gU.sum(0) - 1.0)) < 1e-6
    assert gU.min() >= 0.0 and gU.max() <= 1.0 + 1e-6


def test_phantom1024_matches_oracle(fcm):
    x, _, u0, C = phantom.single_image("phantom1024")
    rep, *_ = paired(fcm, x, C, 2.0, u0=u0, quantized=True)
    assert_within(rep)


@pytest.mark.parametrize("m,recompute,deterministic",
                         [(2.0, False, False), (1.5, False, False), (3.0, False, False), (2.0, True, False),
                          (2.0, False, True)])
def test_volume256_matches_oracle(fcm, m, recompute, deterministic):
    """Full 16.7M-voxel run; U compared on a 200k-voxel sample. By default the
    whole-run kernel hands part of every pass to whichever warps ask first;
    deterministic=True keeps every tile in a fixed warp share."""
    x, _, u0, C = phantom.single_image("volume256")
    kw = dict(recompute=recompute, deterministic=deterministic)
    g, gU, gV = gpu_run(fcm, x, C, m, u0=u0, **kw)
    o = oracle_run(x, C, m, EPS, MAX_ITER, u0=u0, quantized=True, want_U=False)
    assert abs(g.iters - o["iters"]) <= 1
    k = min(g.iters, o["iters"])
    if g.iters > k:
        g, gU, gV = gpu_run(fcm, x, C, m, max_iter=k, u0=u0, **kw)
    if o["iters"] > k:
        o = oracle_run(x, C, m, EPS, k, u0=u0, quantized=True, want_U=False)
    idx = np.random.default_rng(0).choice(x.size, 200_000, replace=False)
    Ubins = oracle.memberships(np.arange(256.0), o["V"], m)
    rep = precision_report(gU[:, idx], gV, g.iters, Ubins[:, x[idx]], o["V"], o["iters"],
                           g.J, o["J"][-1])
    assert_within(rep)


@pytest.mark.parametrize("n,C,m", [(1, 1, 2.0), (3, 2, 2.0), (1001, 3, 1.5), (4099, 5, 3.0),
                                   (65538, 8, 2.0), (123457, 4, 2.7), (40000, 1, 2.0)])
def test_ragged_sizes_match_oracle(fcm, n, C, m):
    side = int(np.ceil(np.sqrt(n)))
    img, _ = phantom.phantom2d(1000 + n, side, side, 9.0)
    x = img.reshape(-1)[:n]
    u0 = phantom.dirichlet_u0((1000 + n, 7), C, n)
    rep, g, *_ = paired(fcm, x, C, m, u0=u0)
    assert_within(rep)


def test_init_from_centers_matches_oracle(fcm):
    x, _, _, C = phantom.single_image("phantom200")
    V0 = np.array([5.0, 45.0, 100.0, 160.0])
    rep, *_ = paired(fcm, x, C, 2.0, V0=V0)
    assert_within(rep)


@pytest.mark.parametrize("k", [7, 30])
def test_max_iter_reached(fcm, k):
    """Stopping at max_iter returns a consistent pair (U^k, V^k) with
    U^k = membership(V^k). Far enough along the trajectory the iterate itself
    matches the oracle's; early on (the symmetry-breaking phase of a random
    start) the map amplifies FP32 rounding, which the per-step test covers."""
    x, _, u0, C = phantom.single_image("phantom200")
    g, gU, gV = gpu_run(fcm, x, C, 2.0, max_iter=k, u0=u0)
    assert g.status == 1 and g.iters == k
    Uo = oracle.memberships(x.astype(np.float64), gV.astype(np.float64), 2.0)
    assert np.max(np.abs(gU - Uo)) <= U_TOL
    if k >= 30:
        o = oracle_run(x, C, 2.0, EPS, k, u0=u0)
        assert o["status"] == oracle.NOT_CONVERGED
        assert_within(precision_report(gU, gV, g.iters, o["U"], o["V"], o["iters"]))


@pytest.mark.parametrize("m", [2.0, 1.5, 3.0, 2.5])
def test_every_iteration_is_one_oracle_step(fcm, m):
    """Each traced iteration of the CUDA run equals one oracle step applied to
    the CUDA run's own centers: U^k = membership(V^k) (Eq. 4), J_k (Eq. 1),
    delta_k = max|U^k - U^{k-1}| and V^{k+1} = centers(U^k) (Eq. 3)."""
    x, _, u0, C = phantom.single_image("phantom200")
    g, _, _ = gpu_run(fcm, x, C, m, u0=u0, trace=True)
    tr = g.trace
    xd = x.astype(np.float64)
    Uprev = u0.astype(np.float64)
    for t in range(g.iters):
        V = tr["V"][t].astype(np.float32).astype(np.float64)  # the centers the pass used
        U = oracle.memberships(xd, V, m)
        J = oracle.objective(xd, U, V, m)
        assert abs(tr["J"][t] - J) <= 1e-5 * J, (t, tr["J"][t], J)
        d = np.max(np.abs(U - Uprev))
        assert abs(tr["delta"][t] - d) <= 1e-6, (t, tr["delta"][t], d)
        if t + 1 < g.iters:
            Vn = oracle.centers(xd, U, m, Vprev=V)[0]
            assert center_err(tr["V"][t + 1], Vn) <= 1e-5, (t, tr["V"][t + 1], Vn)
        Uprev = U
    # J is non-increasing along the CUDA iteration too (FP32 noise allowed)
    assert np.all(np.diff(tr["J"]) <= 1e-6 * tr["J"][0])


@pytest.mark.parametrize("path", ["persistent", "graph", "host_loop", "plain_loads", "recompute"])
@pytest.mark.parametrize("m", [2.0, 3.0, 1.5, 2.5])
def test_every_execution_path_matches_oracle(fcm, path, m):
    """One cooperative launch for the whole run (default), one launch per pass
    in a graph WHILE loop, the host-driven loop, the plain-load kernel, and
    the run that recomputes U^{k-1} instead of storing it."""
    kw = {"persistent": {}, "graph": {"persistent": False}, "host_loop": {"graph": False},
          "plain_loads": {"tma": False}, "recompute": {"recompute": True}}[path]
    x, _, u0, C = phantom.single_image("phantom200")
    g, gU, gV = gpu_run(fcm, x, C, m, u0=u0, **kw)
    o = oracle_run(x, C, m, EPS, MAX_ITER, u0=u0)
    k = min(g.iters, o["iters"])
    d_iters = g.iters - o["iters"]
    if g.iters > k:
        g, gU, gV = gpu_run(fcm, x, C, m, max_iter=k, u0=u0, **kw)
    if o["iters"] > k:
        o = oracle_run(x, C, m, EPS, k, u0=u0)
    assert_within(precision_report(gU, gV, g.iters + d_iters, o["U"], o["V"], o["iters"]))


@pytest.mark.parametrize("n,C", [(4, 2), (132, 3), (1024, 8), (5000, 4), (40960, 5)])
def test_small_aligned_sizes_match_oracle(fcm, n, C):
    """Aligned sizes where warps hold fewer tiles than ring stages (or none)."""
    side = int(np.ceil(np.sqrt(n)))
    img, _ = phantom.phantom2d(2000 + n, side, side, 9.0)
    x = img.reshape(-1)[:n]
    u0 = phantom.dirichlet_u0((2000 + n, 3), C, n)
    rep, *_ = paired(fcm, x, C, 2.0, u0=u0)
    assert_within(rep)
    V0 = np.linspace(10.0, 200.0, C)
    rep, *_ = paired(fcm, x, C, 3.0, V0=V0)
    assert_within(rep)


@pytest.mark.parametrize("n,C", [(4, 2), (132, 3), (1024, 8), (40960, 5), (65536, 1)])
def test_recompute_small_aligned_sizes(fcm, n, C):
    """The recompute run where warps hold fewer tiles than ring stages (or
    none), from U^0 and from centers."""
    side = int(np.ceil(np.sqrt(n)))
    img, _ = phantom.phantom2d(3000 + n, side, side, 9.0)
    x = img.reshape(-1)[:n]
    u0 = phantom.dirichlet_u0((3000 + n, 3), C, n)
    for kw in ({"u0": u0}, {"V0": np.linspace(10.0, 200.0, C)}):
        g, gU, gV = gpu_run(fcm, x, C, 2.0, recompute=True, **kw)
        o = oracle_run(x, C, 2.0, EPS, MAX_ITER, **kw)
        k = min(g.iters, o["iters"])
        d_iters = g.iters - o["iters"]
        if g.iters > k:
            g, gU, gV = gpu_run(fcm, x, C, 2.0, max_iter=k, recompute=True, **kw)
        if o["iters"] > k:
            o = oracle_run(x, C, 2.0, EPS, k, **kw)
        assert_within(precision_report(gU, gV, g.iters + d_iters, o["U"], o["V"], o["iters"]))


def test_recompute_rejects_unaligned_sizes(fcm):
    x, _, u0, C = phantom.single_image("phantom200")
    with pytest.raises(Exception):
        gpu_run(fcm, x[:4001], C, 2.0, u0=u0[:, :4001], recompute=True)


def test_graph_and_host_loop_agree_bitwise(fcm):
    """The per-pass kernels give the same bits from a graph or a host loop."""
    x, _, u0, C = phantom.single_image("phantom200")
    a, aU, aV = gpu_run(fcm, x, C, 2.0, u0=u0, persistent=False)
    b, bU, bV = gpu_run(fcm, x, C, 2.0, u0=u0, graph=False)
    assert a.iters == b.iters and np.array_equal(aU, bU) and np.array_equal(aV, bV)
    assert np.array_equal(a.V64, b.V64)


def test_volume256_runs_repeat(fcm):
    """Two default runs of the volume may round their block sums differently
    (part of every pass goes to whichever warps ask first) and agree to FP32
    rounding; two runs with FCM_OPT_DETERMINISTIC give the same bits."""
    x, _, u0, C = phantom.single_image("volume256")
    a, aU, aV = gpu_run(fcm, x, C, 2.0, u0=u0)
    b, bU, bV = gpu_run(fcm, x, C, 2.0, u0=u0)
    assert abs(a.iters - b.iters) <= 1
    if a.iters == b.iters:
        assert center_err(aV, bV) <= 1e-6 and np.max(np.abs(aU - bU)) <= 1e-6
    del aU, bU
    c, cU, cV = gpu_run(fcm, x, C, 2.0, u0=u0, deterministic=True)
    d, dU, dV = gpu_run(fcm, x, C, 2.0, u0=u0, deterministic=True)
    assert c.iters == d.iters and np.array_equal(cU, dU) and np.array_equal(cV, dV)
    assert np.array_equal(c.V64, d.V64) and c.J == d.J


def test_repeatable(fcm):
    x, _, u0, C = phantom.single_image("phantom200")
    a, aU, aV = gpu_run(fcm, x, C, 3.0, u0=u0)
    b, bU, bV = gpu_run(fcm, x, C, 3.0, u0=u0)
    assert a.iters == b.iters and np.array_equal(aU, bU) and np.array_equal(aV, bV)


def test_host_buffers_match_device_buffers(fcm):
    import torch
    x, _, u0, C = phantom.single_image("phantom200")
    a, aU, aV = gpu_run(fcm, x, C, 2.0, u0=u0)
    xh = torch.from_numpy(x.astype(np.float32)).pin_memory()
    Uh = torch.from_numpy(u0.copy()).pin_memory()
    b = fcm.run(xh, C, 2.0, EPS, MAX_ITER, U=Uh)
    assert b.iters == a.iters and np.array_equal(Uh.numpy(), aU)
    assert np.array_equal(b.V.numpy(), aV)
    # pageable numpy arrays too, with a separate read-only U0
    U0n = u0.copy()
    c = fcm.run(x.astype(np.float32), C, 2.0, EPS, MAX_ITER, U0=U0n)
    assert c.iters == a.iters and np.array_equal(c.U, aU) and np.array_equal(U0n, u0)


def test_separate_u0_is_left_unchanged(fcm):
    x, _, u0, C = phantom.single_image("phantom200")
    a, aU, aV = gpu_run(fcm, x, C, 2.0, u0=u0)
    U0 = _cuda(u0)
    for _ in range(2):
        b = fcm.run(_cuda(x), C, 2.0, EPS, MAX_ITER, U0=U0)
        assert b.iters == a.iters and np.array_equal(b.U.cpu().numpy(), aU)
    assert np.array_equal(U0.cpu().numpy(), u0)


def test_zero_distance_fixed_point(fcm):
    x = np.array([0.0, 10.0] * 64)
    g, gU, gV = gpu_run(fcm, x, 2, 2.0, V0=[0.0, 10.0])
    assert g.status == 0 and g.iters == 1 and g.delta == 0.0
    assert np.array_equal(gV, [0.0, 10.0])
    assert np.array_equal(gU, np.stack([x == 0.0, x == 10.0]).astype(np.float32))


def test_constant_image(fcm):
    """Degenerate image: every center lands exactly on the one grey level (a
    power of two, so the weighted means are exact in any precision), every
    pixel is at distance 0 from all C centers and gets 1/C each."""
    x = np.full(1024, 64.0)
    u0 = phantom.dirichlet_u0((77,), 3, x.size)
    g, gU, gV = gpu_run(fcm, x, 3, 2.0, u0=u0)
    o = oracle_run(x, 3, 2.0, EPS, MAX_ITER, u0=u0)
    assert g.status == 0 and g.iters == o["iters"] == 2
    assert np.array_equal(gV, [64.0, 64.0, 64.0]) and np.array_equal(o["V"], [64.0] * 3)
    assert np.array_equal(gU, np.full((3, 1024), np.float32(1.0) / np.float32(3.0)))


def test_bad_input_is_reported(fcm):
    from paper_1601_00072_gb300 import FcmError
    x, _, u0, C = phantom.single_image("phantom200")
    xb = x.astype(np.float32).copy()
    xb[1234] = np.nan
    with pytest.raises(FcmError) as e:
        gpu_run(fcm, xb, C, 2.0, u0=u0)
    assert e.value.status == -4
    ub = u0.copy()
    ub[2, 77] = -0.25
    with pytest.raises(FcmError) as e:
        gpu_run(fcm, x, C, 2.0, u0=ub)
    assert e.value.status == -4
    with pytest.raises(FcmError) as e:
        gpu_run(fcm, x, C, 2.0, V0=[1.0, np.inf, 3.0, 4.0])
    assert e.value.status == -4
    # the handle stays usable afterwards
    g, *_ = gpu_run(fcm, x, C, 2.0, u0=u0)
    assert g.status == 0


def test_invalid_arguments(fcm):
    import ctypes
    from paper_1601_00072_gb300 import _lib
    L = _lib.load()
    x = _cuda(np.arange(16.0))
    U = _cuda(np.full((2, 16), 0.5))
    V = _cuda(np.zeros(2))
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    h = fcm.handle
    assert L.fcm_run(h, p(x), 16, 2, 1.0, 1e-5, 10, 0, None, p(U), p(V), 0, None) == -1   # m <= 1
    assert L.fcm_run(h, p(x), 16, 0, 2.0, 1e-5, 10, 0, None, p(U), p(V), 0, None) == -1   # C < 1
    assert L.fcm_run(h, p(x), 16, 9, 2.0, 1e-5, 10, 0, None, p(U), p(V), 0, None) == -1   # C > 8
    assert L.fcm_run(h, p(x), 0, 2, 2.0, 1e-5, 10, 0, None, p(U), p(V), 0, None) == -1    # n < 1
    assert L.fcm_run(h, p(x), 16, 2, 2.0, -1.0, 10, 0, None, p(U), p(V), 0, None) == -1   # eps < 0
    assert L.fcm_run(h, p(x), 16, 2, 2.0, 1e-5, 0, 0, None, p(U), p(V), 0, None) == -1    # max_iter
    assert L.fcm_run(h, None, 16, 2, 2.0, 1e-5, 10, 0, None, p(U), p(V), 0, None) == -1   # null x
    assert L.fcm_run(h, p(x), 16, 2, 2.0, 1e-5, 10, 5, None, p(U), p(V), 0, None) == -1   # init mode
    assert L.fcm_run(None, p(x), 16, 2, 2.0, 1e-5, 10, 0, None, p(U), p(V), 0, None) == -1
