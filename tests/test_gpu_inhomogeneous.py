"""The inhomogeneous, time-varying workload (a heated liquid ball in vapour,
periodic box) on the GPU: exact step-0 pair set and forces against the
oracle, and re-tuning between phases without leaving the oracle's FP64
trajectory (every trial step of every phase is a real step, Sec. 1).

A smaller ball (radius 15 in a box of 60, about 13k particles) keeps the
oracle's trajectory within seconds; the full-size scenario (about 292k
particles) is checked at step 0.
"""
import numpy as np
import pytest

import oracle
import paper_2505_03438_gb300 as lj
from paper_2505_03438_gb300 import scenarios

pytestmark = pytest.mark.gpu


def _op(sc):
    return oracle.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], True)


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _wrapdiff(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def _check(s, sc):
    F, e, w = s.compute()
    ref = oracle.forces_cells(_f32(sc["x"]), None, _op(sc), pairs=True)
    pairs, cnt = s.pairs()
    assert cnt == ref["count"]
    assert np.array_equal(oracle.sorted_pairs(pairs), oracle.sorted_pairs(ref["pairs"]))
    assert np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"]) < 1e-5
    assert abs(e - ref["U"]) < 2e-6 * abs(ref["U"])


@pytest.mark.parametrize("cfg", [dict(method="VL"), dict(method="LC", csf=0.5),
                                 dict(method="CL", cluster_size=8, threads_per_unit=8), dict(method="VLW")],
                         ids=["VL", "LC-csf0.5", "CL8", "VLW"])
def test_small_sphere_step0(cfg):
    sc = scenarios.heated_sphere(box_len=60.0, radius=15.0, seed=31)
    s = lj.System(sc)
    s.set_config(rebuild_interval=10, **cfg)
    _check(s, sc)


def test_full_sphere_step0():
    sc = scenarios.heated_sphere()
    assert len(sc["x"]) == 291785 and sc["n_liquid"] == 214466
    s = lj.System(sc)
    _check(s, sc)


@pytest.mark.parametrize("strategy", ["predictive", "expert"])
def test_retuning_phases_stay_on_the_oracle_trajectory(strategy):
    sc = scenarios.heated_sphere(box_len=60.0, radius=15.0, seed=31)
    s = lj.System(sc, precision=1)
    chosen, phases, every = [], 4, 60
    for ph in range(phases):
        c, rep = s.autotune(strategy=strategy, trial_steps=2)
        assert rep["phase"] == ph + 1
        chosen.append(c.name())
        s.step(max(0, every - rep["trial_steps_total"]))
    nsteps = s.counters()["steps"]
    assert nsteps >= every * phases
    x, v = s.state()
    xo, vo, *_ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], _op(sc), sc["dt"], nsteps)
    assert np.abs(_wrapdiff(x, xo, sc["box"][0])).max() < 1e-8, chosen
    assert np.abs(v - vo).max() < 1e-8, chosen


def test_phase_skipped_while_statistics_hold():
    """With skip_within > 0 a phase whose live statistics match those of the
    last phase that ran trials keeps the configuration and runs no trial."""
    sc = scenarios.heated_sphere(box_len=60.0, radius=15.0, seed=31)
    s = lj.System(sc)
    # one trial step per candidate, so that the first phase barely moves the
    # ball and the maximum count per bin (an integer) stays within 10 %
    c1, r1 = s.autotune(strategy="predictive", trial_steps=1, skip_within=0.1)
    assert r1["skipped"] == 0 and r1["ntrialled"] > 0
    steps = s.counters()["steps"]
    c2, r2 = s.autotune(strategy="predictive", trial_steps=1, skip_within=0.1)
    assert r2["skipped"] == 1 and r2["ntrialled"] == 0 and r2["phase"] == r1["phase"]
    assert c2.name() == c1.name() and s.counters()["steps"] == steps
    c3, r3 = s.autotune(strategy="predictive", trial_steps=1, skip_within=0.0)
    assert r3["skipped"] == 0 and r3["phase"] == r1["phase"] + 1


def test_tuning_cost_uses_the_observed_rebuild_interval():
    """When most rebuilds since the last phase came early (a particle reached
    skin/2 before R steps), the next phase weights build times by the
    observed steps per rebuild instead of R (reported as rebuild_every)."""
    sc = scenarios.heated_sphere(box_len=60.0, radius=15.0, seed=31)
    s = lj.System(sc)
    _, r1 = s.autotune(strategy="full", trial_steps=2)
    assert r1["rebuild_every"] == 0.0  # no window yet
    c1 = s.counters()
    s.step(200)
    c2 = s.counters()
    dr, de = c2["rebuilds"] - c1["rebuilds"], c2["early_rebuilds"] - c1["early_rebuilds"]
    _, r2 = s.autotune(strategy="full", trial_steps=2)
    assert dr > 0 and 2 * de >= dr, (dr, de)  # the hot ball forces early rebuilds
    assert abs(r2["rebuild_every"] - 200.0 / dr) < 1e-9, (r2["rebuild_every"], dr)
    assert 0.0 < r2["rebuild_every"] < 20.0
    s.close()
