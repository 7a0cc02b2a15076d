"""Host-side logic of the warm start (CPU only): the acceptance rule of a
warm-started slice against its cold start, and the keys of the random starts."""
from types import SimpleNamespace

import numpy as np

import phantom
from paper_1601_00072_gb300 import warmstart


def _run(V, J, status=0):
    V = np.asarray(V, dtype=np.float64)
    V64 = np.zeros(8)
    V64[:V.size] = V
    return SimpleNamespace(C=V.size, V64=V64, J=J, status=status)


def test_same_centers_in_any_order_are_accepted():
    cold = _run([10.0, 80.0, 150.0], 100.0)
    warm = _run([150.0, 10.0, 80.0 * (1 + 5e-5)], 100.5)  # J larger, centers equal within 1e-4
    assert warmstart.accepted([cold], [warm]).tolist() == [True]


def test_center_error_is_relative_to_max_of_v_and_one():
    # |dv| / max(|v|, 1): near 0 the tolerance is absolute 1e-4
    cold = _run([0.2, 50.0], 10.0)
    assert warmstart.accepted([cold], [_run([0.2 + 9e-5, 50.0], 11.0)]).tolist() == [True]
    assert warmstart.accepted([cold], [_run([0.2 + 2e-4, 50.0], 11.0)]).tolist() == [False]


def test_other_minimum_with_no_larger_objective_is_accepted():
    cold = _run([20.0, 90.0, 160.0], 1000.0)
    lower = _run([25.0, 95.0, 170.0], 990.0)
    within_slack = _run([25.0, 95.0, 170.0], 1000.0 * (1 + 0.9e-5))
    higher = _run([25.0, 95.0, 170.0], 1000.0 * (1 + 2e-5))
    assert warmstart.accepted([cold] * 3, [lower, within_slack, higher]).tolist() == [True, True, False]


def test_failed_warm_run_is_not_accepted_on_its_objective():
    cold = _run([20.0, 90.0], 500.0)
    failed = _run([30.0, 99.0], 100.0, status=-4)
    assert warmstart.accepted([cold], [failed]).tolist() == [False]


def test_start_keys_are_distinct_and_start_zero_is_the_batch_key():
    keys = {warmstart.u0_key(i, s) for i in range(64) for s in range(warmstart.STARTS)}
    assert len(keys) == 64 * warmstart.STARTS
    assert warmstart.u0_key(7, 0) == (phantom.U0_FAMILY, 7)
    # the drawn memberships differ between starts and are valid columns
    a = phantom.dirichlet_u0(warmstart.u0_key(3, 0), 4, 100)
    b = phantom.dirichlet_u0(warmstart.u0_key(3, 1), 4, 100)
    assert not np.array_equal(a, b)
    assert np.allclose(a.sum(0), 1.0, atol=1e-6) and (a >= 0).all()
