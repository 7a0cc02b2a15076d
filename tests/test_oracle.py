"""The FP64 oracle holds every pin (CPU only)."""
import numpy as np
import pytest

import oracle_pins
from oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda p: p.__name__)
def test_pin_holds(orc, pin):
    fails = pin(orc.lib())
    assert not fails, "\n".join(fails)


def test_rejects_bad_arguments(orc):
    x = np.arange(10.0)
    with pytest.raises(ValueError):
        orc.fcm(x, 2, 1.0, 1e-5, 10, V0=[1.0, 2.0])      # m must exceed 1
    with pytest.raises(ValueError):
        orc.fcm(x, 2, 2.0, 1e-5, 0, V0=[1.0, 2.0])       # max_iter >= 1
    with pytest.raises(ValueError):
        orc.fcm(x, 2, 2.0, -1.0, 10, V0=[1.0, 2.0])      # eps >= 0


def test_not_converged_status(orc):
    import phantom
    img, _ = phantom.phantom2d(5, 32, 32, 8.0)
    x = img.reshape(-1).astype(float)
    r = orc.fcm(x, 4, 2.0, 1e-12, 3, U0=phantom.dirichlet_u0((5, 1), 4, x.size))
    assert r["status"] == orc.NOT_CONVERGED and r["iters"] == 3
