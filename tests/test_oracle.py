"""The FP64 oracle against its pins (CPU only)."""
import numpy as np
import pytest

import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc.load())


def test_scenarios_state_point():
    from paper_2505_03438_gb300 import scenarios
    sc = scenarios.small_fcc()
    n = len(sc["x"])
    assert n == 4000
    assert abs(n / np.prod(sc["box"]) - 0.8442) < 1e-12
    v = sc["v"]
    assert np.abs(v.sum(0)).max() < 1e-12
    t = (v * v).sum() / (3 * n - 3)
    assert abs(t - 0.72) < 1e-12
    mix = scenarios.binary_mixture()
    assert len(mix["x"]) == 32768 and int((mix["types"] == 0).sum()) == 26214
    assert abs(32768 / np.prod(mix["box"]) - 1.2) < 1e-12
    assert np.allclose(mix["rcut"], 2.5 * mix["sigma"])
