"""Pair sets and forces after real dynamics, not only at step 0: the
full-size liquid (N = 1,048,576) after 500 and 1000 steps in the
benchmark's launch configuration, the heated sphere (about 292k particles)
after 1000 steps, and sampled replicas of the 512-replica batch after 200
steps.  At each snapshot the oracle works on the positions the GPU's pair
arithmetic used (the working-precision copy promoted exactly to double,
unwrapped, as between rebuilds); pair sets must be equal bit for bit and
forces within 1e-5 relative RMS."""
import numpy as np
import pytest

import oracle
import paper_2505_03438_gb300 as lj
from paper_2505_03438_gb300 import scenarios

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _op(sc):
    return oracle.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], sc.get("shift", True))


def _snapshot(s, sc):
    xw = s.work_positions()
    F, e, w = s.compute()
    pairs, cnt = s.pairs()
    ref = oracle.forces_cells(xw, sc["types"], _op(sc), pairs=True)
    assert cnt == ref["count"], (cnt, ref["count"])
    assert np.array_equal(oracle.sorted_pairs(pairs), oracle.sorted_pairs(ref["pairs"]))
    assert np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"]) <= 1e-5
    assert abs(e - ref["U"]) <= 1e-5 * abs(ref["U"])
    assert abs(w - ref["W"]) <= 1e-5 * abs(ref["W"])
    return cnt


def test_liquid_1m_after_500_and_1000_steps():
    sc = scenarios.liquid_1m()
    s = lj.System(sc)
    s.set_config(method="VL", threads_per_unit=2, rebuild_interval=10)
    counts = []
    for k in (500, 500):
        s.step(k)
        counts.append(_snapshot(s, sc))
    c = s.counters()
    assert c["steps"] == 1000 and c["rebuilds"] >= 50  # the lists were rebuilt many times on the way
    # the melting lattice changes its neighbourhoods: the pair sets differ
    assert counts[0] != counts[1]
    s.close()


def test_heated_sphere_after_1000_steps():
    sc = scenarios.heated_sphere()
    s = lj.System(sc)
    s.set_config(method="VL", threads_per_unit=2, rebuild_interval=10)
    s.step(1000)
    _snapshot(s, sc)
    s.close()


def test_replica_batch_after_200_steps_sampled():
    reps = scenarios.replica_batch()
    b = lj.Batch(reps)
    b.step(200)
    xw = b.split(b.work_positions())
    F, e, w = b.compute()
    Fr = b.split(F)
    pairs = b.pairs()
    counts = np.array([len(r["x"]) for r in reps])
    rng = np.random.default_rng(57)
    pick = sorted(set([int(counts.argmin()), int(counts.argmax())] + rng.choice(len(reps), 8, replace=False).tolist()))
    for r in pick:
        sc = reps[r]
        ref = oracle.forces_cells(xw[r], None, _op(sc), pairs=True)
        mine = pairs[pairs[:, 0] == r][:, 1:]
        assert np.array_equal(oracle.sorted_pairs(mine), oracle.sorted_pairs(ref["pairs"])), r
        assert np.linalg.norm(Fr[r] - ref["F"]) / np.linalg.norm(ref["F"]) <= 1e-5, r
        assert abs(e[r] - ref["U"]) <= 1e-5 * abs(ref["U"]), r
    b.close()
