"""Pins of the counter-based initial membership (CPU only).

The library can draw the random U^0 of Algorithm 1 step 2 on the device
(fcm_init_dirichlet). Its definition, Philox4x32-10 turned into a uniform
Dirichlet(1, ..., 1) per pixel, is implemented a second time in the input
generator module (``phantom.philox_dirichlet_u0``), which the GPU tests
compare with. Here that host implementation is pinned to the generator's
published known-answer vectors and to the moments of the distribution.
"""
import json
import os

import numpy as np
import pytest

import phantom

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.json")


def test_philox_known_answers():
    for v in json.load(open(GOLDEN))["vectors"]:
        ctr = [[int(c, 16)] for c in v["ctr"]]
        key = tuple(int(k, 16) for k in v["key"])
        out = phantom.philox4x32_10(ctr, key)
        assert [int(o[0]) for o in out] == [int(w, 16) for w in v["out"]]


def test_philox_is_a_function_of_counter_and_key():
    a = phantom.philox4x32_10([np.arange(8), np.zeros(8), np.zeros(8), np.zeros(8)], (7, 9))
    b = phantom.philox4x32_10([np.arange(8)[::-1], np.zeros(8), np.zeros(8), np.zeros(8)], (7, 9))
    for wa, wb in zip(a, b):
        assert np.array_equal(wa, wb[::-1])
    c = phantom.philox4x32_10([np.arange(8), np.zeros(8), np.zeros(8), np.zeros(8)], (7, 10))
    assert not np.array_equal(a[0], c[0])


@pytest.mark.parametrize("C", [1, 3, 4, 5, 8])
def test_dirichlet_moments(C):
    """Each column sums to 1; a uniform Dirichlet(1, ..., 1) has marginals
    Beta(1, C - 1): mean 1/C, E[u^2] = 2 / (C (C + 1)). Checked at 5 standard
    errors on 200,000 pixels."""
    n = 200_000
    U = phantom.philox_dirichlet_u0(12345, C, n).astype(np.float64)
    assert U.shape == (C, n) and U.dtype == np.float64
    assert np.max(np.abs(U.sum(0) - 1.0)) < 1e-6
    assert U.min() >= 0.0
    if C == 1:
        assert np.all(U == 1.0)
        return
    m1, m2 = 1.0 / C, 2.0 / (C * (C + 1))
    var1 = m2 - m1 ** 2
    m4 = 24.0 / (C * (C + 1) * (C + 2) * (C + 3))  # E[u^4] of Beta(1, C - 1)
    for j in range(C):
        assert abs(U[j].mean() - m1) < 5 * np.sqrt(var1 / n)
        assert abs((U[j] ** 2).mean() - m2) < 5 * np.sqrt((m4 - m2 ** 2) / n)


def test_dirichlet_blocks_and_seed():
    """Clusters 0..3 use block 0 of the counter and clusters 4..7 block 1, so
    the first four clusters' exponentials do not depend on C beyond 4; another
    seed gives another draw."""
    a = phantom.philox_dirichlet_u0(5, 8, 1000).astype(np.float64)
    b = phantom.philox_dirichlet_u0(5, 4, 1000).astype(np.float64)
    # u_j = E_j / sum E: the ratios u_0 / u_1 agree between C = 8 and C = 4
    assert np.allclose(a[0] / a[1], b[0] / b[1], rtol=1e-6)
    assert not np.allclose(phantom.philox_dirichlet_u0(6, 4, 1000), b)
