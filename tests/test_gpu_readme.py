"""The usage shown at the top of the package's documentation, run as
written (a small fcc liquid, the shipped forest, 1000 steps), with its
results checked against the oracle."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_documented_usage_runs_and_is_right():
    import paper_2505_03438_gb300 as lj
    from paper_2505_03438_gb300 import scenarios

    sc = scenarios.fcc_liquid(20)
    s = lj.System(sc)
    s.set_forest()
    cfg, report = s.autotune(strategy="forest")
    s.step(1000)
    F, epot, virial = s.compute()
    x, v = s.state()
    assert report["ntrialled"] in (0, 1) and cfg.name() == s.config().name()
    assert x.shape == (32000, 3) and np.isfinite(x).all() and (x >= 0).all() and (x < sc["box"][0]).all()
    # forces and energy at the final positions, as the oracle computes them
    ref = oracle.forces_cells(s.work_positions(), None,
                              oracle.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], True))
    assert np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"]) <= 1e-5
    assert abs(epot - ref["U"]) <= 1e-5 * abs(ref["U"])
    s.close()
