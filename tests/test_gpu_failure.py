"""Failure detection and resumption, without faulting the GPU.

* A bounded device wait on a flag that nothing sets gives up and the host
  reads LJSEL_ERR_TIMEOUT; the context stays usable afterwards.
* Non-finite input (injected on the host) is reported as
  LJSEL_ERR_NONFINITE by the device flags, never trapped.
* A checkpoint written to .npz resumes the FP64 trajectory.
* Particle types outside the parameter table are refused at creation.
"""
import numpy as np
import pytest

import oracle
import paper_2505_03438_gb300 as lj
from paper_2505_03438_gb300 import scenarios

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    assert lj.ljsel_selftest_wait_timeout(1 << 14) == 7  # LJSEL_ERR_TIMEOUT
    assert "bounded device wait" in lj.ljsel_last_error()
    # the GPU still works: a small system steps and matches the oracle's forces
    sc = scenarios.fcc_liquid(4, seed=3, jitter=0.1)
    s = lj.System(sc, precision=1)
    F, _, _ = s.compute()
    ref = oracle.forces_cells(sc["x"], None, oracle.make_params(sc["box"], 1.0, 1.0, 2.5, True))
    assert np.abs(F - ref["F"]).max() < 1e-11 * np.abs(ref["F"]).max()


@pytest.mark.parametrize("where", ["position", "velocity"])
def test_nonfinite_input_is_reported(where):
    sc = scenarios.fcc_liquid(4, seed=5, jitter=0.1)
    x, v = sc["x"].copy(), sc["v"].copy()
    (x if where == "position" else v)[7, 1] = np.nan
    s = lj.System(sc)
    s.set_state(x, v)
    with pytest.raises(lj.LjselError) as e:
        s.step(5)
    assert e.value.status == 6  # LJSEL_ERR_NONFINITE


def test_checkpoint_resumes_the_trajectory(tmp_path):
    sc = scenarios.fcc_liquid(5, seed=9, jitter=0.1)
    a = lj.System(sc, precision=1)
    a.set_config(method="VL", rebuild_interval=7)
    a.step(30)
    path = str(tmp_path / "ck.npz")
    a.checkpoint(path)
    a.step(25)
    xa, va = a.state()
    b = lj.System.from_checkpoint(path)
    assert b.config().name() == a.config().name()
    b.step(25)
    xb, vb = b.state()
    L = sc["box"][0]
    d = xa - xb
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-10 and np.abs(va - vb).max() < 1e-10


@pytest.mark.parametrize("bad", [2, -1])
def test_types_outside_the_table_are_refused(bad):
    """The import kernel checks every type against [0, ntypes); the creating
    call reports LJSEL_ERR_ARG and frees what it allocated."""
    sc = scenarios.binary_mixture(seed=14, nside=7)
    t = np.asarray(sc["types"], np.int32).copy()
    t[len(t) // 2] = bad
    with pytest.raises(lj.LjselError) as e:
        lj.System(dict(sc, types=t))
    assert e.value.status == 1 and "ntypes" in lj.ljsel_last_error()
    s = lj.System(sc)  # the valid input still works
    s.compute()
    s.close()
