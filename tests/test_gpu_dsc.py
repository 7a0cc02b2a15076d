"""The CUDA defuzzification + Dice score (fcm_dsc) against the oracle's
definition of Eq. 5 (needs a GPU)."""
import numpy as np
import pytest

import oracle
import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fcm():
    from paper_1601_00072_gb300 import _build
    _build.build()
    from paper_1601_00072_gb300.fcm import FCM
    h = FCM(0)
    yield h
    h.close()


def _cuda(a, dtype=np.float32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


@pytest.mark.parametrize("n,C,K", [(1, 1, 1), (1000, 3, 3), (65537, 4, 4), (300001, 8, 5)])
def test_counts_are_exact(fcm, n, C, K):
    """Memberships drawn by the test (with exact ties), so both sides score
    the same U: the counts and scores must be identical."""
    g = np.random.default_rng(n)
    U = g.random((C, n)).astype(np.float32)
    tie = g.random(n) < 0.1
    U[:, tie] = 0.5  # every cluster ties: label 0
    truth = g.integers(0, K, n).astype(np.uint8)
    cmap = g.integers(0, K, C).astype(np.int32)
    d, c = fcm.dsc(_cuda(U), _cuda(truth, np.uint8), K, class_of_cluster=cmap)
    od, oc = oracle.dsc(oracle.labels(U.astype(np.float64)), truth, cmap, K)
    assert np.array_equal(c, oc)
    assert np.array_equal(d, od)


def test_fcm_segmentation_of_the_phantom(fcm):
    """The CUDA run's segmentation scored on the CUDA side equals the oracle
    run's scored by the oracle, to the label agreement of the two runs."""
    x, lab, u0, C = phantom.single_image("phantom200")
    r = fcm.run(_cuda(x), C, 2.0, 1e-5, 300, U0=_cuda(u0))
    d, _ = fcm.dsc(r.U, _cuda(lab, np.uint8), C, V=r.V)
    o = oracle.fcm(x.astype(np.float64), C, 2.0, float(np.float32(1e-5)), 300, U0=u0)
    cmap = np.empty(C, dtype=np.int32)
    cmap[np.argsort(o["V"])] = np.arange(C)
    od, _ = oracle.dsc(oracle.labels(o["U"]), lab, cmap, C)
    assert np.max(np.abs(d - od)) <= 1e-3
    assert np.all(d > 0.5)  # the phantom's four tissues are found


def test_truth_out_of_range_is_rejected(fcm):
    U = np.full((2, 10), 0.5, dtype=np.float32)
    truth = np.zeros(10, dtype=np.uint8)
    truth[3] = 7
    with pytest.raises(Exception):
        fcm.dsc(_cuda(U), _cuda(truth, np.uint8), 2, class_of_cluster=[0, 1])
