"""Reflective walls and the velocity-scaling thermostat on the GPU against
the FP64 oracle (the walled heating-sphere conditions of Sec. 6).

Between walls a dimension has no periodic image, and a particle that
crosses a wall after a drift is mirrored back with its velocity component
reversed.  Walls are available with the linked-cell, Verlet-list and
cluster-list methods.
"""
import numpy as np
import pytest

import oracle
import paper_2505_03438_gb300 as lj
from paper_2505_03438_gb300 import scenarios

pytestmark = pytest.mark.gpu

CONFIGS = [dict(method="LC"), dict(method="LC", newton3=True), dict(method="LC", csf=0.5),
           dict(method="VL"), dict(method="VL", threads_per_unit=4), dict(method="VL", newton3=True),
           dict(method="VL", csf=0.5), dict(method="VL", newton3=True, csf=0.5),
           dict(method="CL", cluster_size=4, threads_per_unit=8), dict(method="CL", cluster_size=2, threads_per_unit=2),
           dict(method="CL", cluster_size=8, newton3=True, threads_per_unit=8),
           dict(method="CL", cluster_size=4, newton3=True, threads_per_unit=4, csf=0.5)]


def _gas(seed, L=11.0, n=500):
    """A random gas with some particles moved onto or next to a face (step-0
    checks only: the moved particles may overlap)."""
    sc = scenarios.random_gas(n, L, seed=seed, min_dist=0.85)
    # crowd some particles against the faces
    x = sc["x"]
    near = np.arange(0, n, 7)
    x[near, seed % 3] = np.where(x[near, seed % 3] < L / 2, 0.02 * (near % 5), L - 0.02 * (near % 5))
    return sc


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


@pytest.mark.parametrize("walls", [(1, 1, 1), (1, 0, 0), (0, 1, 1)], ids=["xyz", "x", "yz"])
@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "-".join("%s%s" % kv for kv in c.items()))
def test_pairs_and_forces_with_walls(walls, cfg):
    for precision in (0, 1):
        sc = _gas(31 + sum(walls))
        s = lj.System(sc, walls=walls, precision=precision)
        s.set_config(rebuild_interval=10, **cfg)
        F, e, w = s.compute()
        xo = sc["x"] if precision else _f32(sc["x"])
        p = oracle.make_params(sc["box"], 1.0, 1.0, 2.5, True, walls=walls)
        ref = oracle.forces_cells(xo, None, p, pairs=True)
        pairs, cnt = s.pairs()
        assert cnt == ref["count"]
        assert np.array_equal(oracle.sorted_pairs(pairs), oracle.sorted_pairs(ref["pairs"]))
        tol = 1e-12 if precision else 1e-5
        assert np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"]) < tol
        assert abs(e - ref["U"]) < max(tol, 2e-6) * abs(ref["U"])


@pytest.mark.parametrize("method", ["LC", "VL", "CL"])
def test_walled_liquid_trajectory_fp64(method):
    x, box = scenarios.fcc_lattice(4, 0.7)
    L = box[0] + 1.0
    x = x + 0.5
    rng = np.random.default_rng(41)
    v = scenarios.maxwell_boltzmann(len(x), 1.5, 1.0, rng)
    s = lj.System(x=x, v=v, box=np.full(3, L), walls=(1, 1, 1), precision=1, dt=0.002)
    s.set_config(method=method, rebuild_interval=10, **(dict(cluster_size=4, threads_per_unit=8) if method == "CL" else {}))
    s.step(300)
    xg, vg = s.state()
    p = oracle.make_params(L, 1.0, 1.0, 2.5, True, walls=(1, 1, 1))
    xo, vo, *_ = oracle.verlet_run(x, v, None, [1.0], p, 0.002, 300)
    assert np.abs(xg - xo).max() < 1e-9 and np.abs(vg - vo).max() < 1e-9
    assert xg.min() >= 0.0 and xg.max() <= L


def test_free_particles_bounce():
    L, dt, nsteps = 8.0, 0.01, 611
    x0 = np.array([[1.0, 7.5, 3.0], [6.0, 1.0, 1.0]])
    v0 = np.array([[1.3, 0.7, -2.9], [-0.4, 2.2, 0.1]])
    s = lj.System(x=x0, v=v0, box=np.full(3, L), walls=(1, 1, 1), precision=1, dt=dt, skin=0.3)
    s.set_config(method="LC", rebuild_interval=1)
    s.step(nsteps)
    x, v = s.state()
    u = x0 + v0 * dt * nsteps
    k = np.floor(u / L)
    assert np.abs(x - np.where(k % 2 == 0, u - k * L, (k + 1) * L - u)).max() < 1e-9
    assert np.allclose(v, np.where(k % 2 == 0, v0, -v0))


@pytest.mark.parametrize("walls", [(0, 0, 0), (1, 1, 1)], ids=["periodic", "walls"])
def test_thermostat_matches_the_oracle(walls):
    sc = scenarios.fcc_liquid(5, seed=43, jitter=0.05)
    L = sc["box"][0]
    s = lj.System(sc, walls=walls, precision=1)
    _, v = s.state()
    p = oracle.make_params(L, 1.0, 1.0, 2.5, True, walls=walls)
    v_ref, t_ref = oracle.thermostat(v, None, [1.0], p, 2.0, 0.1)
    t = s.thermostat(2.0, 0.1)
    _, v2 = s.state()
    assert abs(t - t_ref) < 1e-12 * t_ref
    assert np.abs(v2 - v_ref).max() < 1e-12 * np.abs(v_ref).max()


HEAT_CFGS = [dict(method="VL"), dict(method="VL", newton3=True), dict(method="LC"), dict(method="LC", newton3=True),
             dict(method="CL", cluster_size=4, threads_per_unit=4),
             dict(method="CL", cluster_size=2, newton3=True, threads_per_unit=4)]


@pytest.mark.parametrize("cfg", HEAT_CFGS, ids=lambda c: "-".join("%s%s" % kv for kv in c.items()))
def test_heating_in_walls_follows_the_oracle_fp64(cfg):
    """A small walled heating run for every method that supports walls:
    every 50 steps the temperature moves by at most 0.1 towards 3.0 (the
    heating-sphere protocol of Sec. 6, scaled down); the FP64 trajectory
    stays on the oracle's."""
    x, box = scenarios.fcc_lattice(3, 0.75)
    L = box[0] + 4.0
    x = x + 2.0
    rng = np.random.default_rng(44)
    v = scenarios.maxwell_boltzmann(len(x), 0.7, 1.0, rng)
    s = lj.System(x=x, v=v, box=np.full(3, L), walls=(1, 1, 1), precision=1, dt=0.002)
    s.set_config(rebuild_interval=10, **cfg)
    p = oracle.make_params(L, 1.0, 1.0, 2.5, True, walls=(1, 1, 1))
    xo, vo = x.copy(), v.copy()
    temps = []
    for _ in range(6):
        s.step(50)
        temps.append(s.thermostat(3.0, 0.1))
        xo, vo, *_ = oracle.verlet_run(xo, vo, None, [1.0], p, 0.002, 50)
        vo, _ = oracle.thermostat(vo, None, [1.0], p, 3.0, 0.1)
    xg, vg = s.state()
    assert np.abs(xg - xo).max() < 1e-8 and np.abs(vg - vo).max() < 1e-8
    assert temps[-1] > temps[0]


def test_walled_heating_sphere_workload_step0():
    """The walled heating sphere of Sec. 6 (5497 particles, cutoff 3, skin
    0.5): pair set and FP32 forces against the oracle at the start, for the
    linked-cell, Verlet-list and cluster-list methods."""
    sc = scenarios.walled_heating_sphere()
    p = oracle.make_params(sc["box"], 1.0, 1.0, 3.0, True, walls=(1, 1, 1))
    ref = oracle.forces_cells(_f32(sc["x"]), None, p, pairs=True)
    for cfg in (dict(method="LC"), dict(method="VL"), dict(method="CL", cluster_size=4, threads_per_unit=8)):
        s = lj.System(sc)
        s.set_config(rebuild_interval=10, **cfg)
        F, e, w = s.compute()
        pairs, cnt = s.pairs()
        assert cnt == ref["count"]
        assert np.array_equal(oracle.sorted_pairs(pairs), oracle.sorted_pairs(ref["pairs"]))
        assert np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"]) < 1e-5
        assert abs(e - ref["U"]) < 2e-6 * abs(ref["U"])
        s.close()


def test_walls_with_window_lists_are_refused():
    sc = scenarios.random_gas(500, 11.0, seed=35, min_dist=0.85)
    s = lj.System(sc, walls=(1, 1, 1))
    with pytest.raises(lj.LjselError) as e:
        s.set_config(method="VLW")
    assert e.value.status == 9
    chosen, rep = s.autotune(strategy="full", trial_steps=2)
    assert chosen.method in (lj.METHOD_LC, lj.METHOD_VL, lj.METHOD_CLUSTER)
