"""The on-device random start (fcm_init_dirichlet, fcm_run_seeded) against
its host implementation and the FP64 oracle (needs a GPU).

The library draws U^0 from Philox4x32-10 with FP32 logarithms; the input
generator module implements the same definition in FP64
(``phantom.philox_dirichlet_u0``, pinned to the generator's known answers).
The integer streams are the same, so the two U^0 agree to FP32 rounding; a
run from the device start matches the oracle run from the host start."""
import numpy as np
import pytest

import oracle
import phantom
from parity import assert_within, eps32, precision_report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fcm():
    from paper_1601_00072_gb300 import _build
    _build.build()
    from paper_1601_00072_gb300.fcm import FCM
    h = FCM(0)
    yield h
    h.close()


@pytest.mark.parametrize("C,n,seed", [(1, 1, 3), (3, 1001, 7), (4, 65536, 2 ** 40 + 17), (5, 4097, 0),
                                      (8, 300_000, 123456789)])
def test_device_start_equals_host_definition(fcm, C, n, seed):
    U = fcm.init_dirichlet(n, C, seed).cpu().numpy().astype(np.float64)
    ref = phantom.philox_dirichlet_u0(seed, C, n).astype(np.float64)
    assert np.max(np.abs(U - ref)) <= 1e-6
    assert np.max(np.abs(U.sum(0) - 1.0)) <= 1e-6 and U.min() >= 0.0


def test_seeded_run_matches_oracle(fcm):
    """Both sides at the same iterate: the longer run is repeated with
    max_iter equal to the shorter count."""
    import torch
    x, _, _, C = phantom.single_image("phantom200")
    seed = 101
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    x64 = x.astype(np.float64)
    u0 = phantom.philox_dirichlet_u0(seed, C, x.size)
    g = fcm.run_seeded(xt, C, 2.0, 1e-5, 300, seed=seed)
    o = oracle.fcm(x64, C, 2.0, eps32(1e-5), 300, U0=u0)
    d_iters = g.iters - o["iters"]
    k = min(g.iters, o["iters"])
    if g.iters > k:
        g = fcm.run_seeded(xt, C, 2.0, 1e-5, k, seed=seed)
    if o["iters"] > k:
        o = oracle.fcm(x64, C, 2.0, 0.0, k, U0=u0)
    rep = precision_report(g.U.cpu().numpy(), g.V.cpu().numpy(), k + d_iters, o["U"], o["V"], k)
    assert_within(rep)
