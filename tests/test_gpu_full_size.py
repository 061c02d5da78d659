"""Every configuration the tuner can choose, at the benchmark's full size,
against the FP64 oracle (Sec. 2.1 forces over the traversals of Sec. 2.2.1).

The homogeneous liquid of N = 1,048,576 (fcc 64^3 x 4, rho 0.8442): each
default candidate builds its neighbour structure at the lattice positions,
the particles are then moved by generator-made displacements below skin/2
(the structure is kept, as between rebuilds), and the pair set (bit-exact)
and the FP32 forces (1e-5 relative RMS), energy and virial (2e-6) are
compared with one oracle evaluation at those positions.  This covers the
full-size values of every capacity, stride and index a configuration uses
(list rows, cluster counts, the 27-bit list index, the cell grids of CSF 1
and 0.5).  The heated sphere (291,785 particles) is checked the same way at
step 0 for cluster and linked-cell configurations.
"""
import numpy as np
import pytest

import oracle
from paper_2505_03438_gb300 import scenarios

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
SUM_TOL = 2e-6


@pytest.fixture(scope="module")
def lj():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_03438_gb300 as m
    return m


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _keys(pairs, n):
    """Sorted int64 keys lo * n + hi of an unordered pair array."""
    p = np.asarray(pairs, np.int64).reshape(-1, 2)
    lo = np.minimum(p[:, 0], p[:, 1])
    hi = np.maximum(p[:, 0], p[:, 1])
    return np.sort(lo * n + hi)


def _drift(x, box, seed, amp):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=x.shape)
    d *= (amp * rng.uniform(0.2, 1.0, (len(x), 1))) / np.linalg.norm(d, axis=1, keepdims=True)
    return x + d


def _check(s, sc, ref, keys_ref, n):
    F, e, w = s.compute()
    pairs, cnt = s.pairs()
    assert cnt == ref["count"], (cnt, ref["count"])
    assert np.array_equal(_keys(pairs, n), keys_ref)
    rel = np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"])
    assert rel <= FORCE_TOL, rel
    assert abs(e - ref["U"]) <= SUM_TOL * abs(ref["U"]), (e, ref["U"])
    assert abs(w - ref["W"]) <= SUM_TOL * abs(ref["W"]), (w, ref["W"])
    return rel


def test_every_candidate_liquid_1m(lj):
    sc = scenarios.liquid_1m()
    n = len(sc["x"])
    x1 = _drift(sc["x"], sc["box"], 91, 0.9 * 0.5 * sc["skin"])
    p = oracle.make_params(sc["box"], 1.0, 1.0, 2.5, True)
    ref = oracle.forces_cells(_f32(x1), None, p, pairs=True)
    keys_ref = _keys(ref["pairs"], n)
    s = lj.System(sc)
    cands = lj.ljsel_default_candidates(s.h)
    names = [c.name() for c in cands]
    assert any(nm.startswith("CL") for nm in names) and any(nm.startswith("LC") for nm in names)
    checked = []
    for c in cands:
        s.set_state(sc["x"], sc["v"])
        lj.ljsel_set_config(s.h, c)
        s.compute()  # the structure of this configuration, built at the lattice positions
        nreb = s.counters()["rebuilds"]
        s.move_particles(x1)
        _check(s, sc, ref, keys_ref, n)
        assert s.counters()["rebuilds"] == nreb, c.name()  # the lattice build was used
        checked.append(c.name())
    assert checked == names


@pytest.mark.parametrize("cfg", [dict(method="CL", cluster_size=4, threads_per_unit=4),
                                 dict(method="CL", cluster_size=2, newton3=True, threads_per_unit=4),
                                 dict(method="LC", newton3=True), dict(method="LC", csf=0.5)],
                         ids=["CL4", "CL2-N3L", "LC-N3L", "LC-csf0.5"])
def test_heated_sphere_step0(lj, cfg):
    sc = scenarios.heated_sphere()
    n = len(sc["x"])
    p = oracle.make_params(sc["box"], 1.0, 1.0, 2.5, True)
    ref = oracle.forces_cells(_f32(sc["x"]), None, p, pairs=True)
    s = lj.System(sc)
    s.set_config(rebuild_interval=10, **cfg)
    _check(s, sc, ref, _keys(ref["pairs"], n), n)
    s.close()
