"""Batched replicas on the GPU against the FP64 oracle, replica by replica.

Inputs are the seeded generator's replicas (N log-uniform, density U[0.3,
0.9], T U[0.7, 2.0], jittered cubic lattices).  The oracle sees only
generator data: at step 0 the positions the FP32 pair arithmetic uses are
the generator's positions rounded to float32 (done here in numpy); after
steps the FP64 batch is compared with the oracle's own trajectories.
"""
import numpy as np
import pytest

import oracle
import paper_2505_03438_gb300 as lj
from paper_2505_03438_gb300 import scenarios

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5


def _op(sc):
    return oracle.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], True)


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _wrapdiff(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def _small_batch(seed=41, nrep=24):
    return scenarios.replica_batch(nrep=nrep, seed=seed, nmin=256, nmax=1500)


def _edge_batch():
    """Ragged edges: an empty replica, a two-particle replica with no pair in
    range, the smallest box the cell grid allows (2 cells per side)."""
    reps = _small_batch(seed=43, nrep=3)
    box = np.full(3, 5.7)
    empty = dict(reps[0], x=np.zeros((0, 3)), v=np.zeros((0, 3)), types=np.zeros(0, np.int32), box=box)
    two = dict(reps[0], x=np.array([[0.5, 0.5, 0.5], [3.3, 3.3, 3.3]]), v=np.array([[0.1, 0, 0], [-0.1, 0, 0]]),
               types=np.zeros(2, np.int32), box=box)
    return [reps[0], empty, reps[1], two, reps[2]]


def _check_step0(b, reps, precision, force_tol):
    F, e, w = b.compute()
    pairs = b.pairs()
    Fr = b.split(F)
    for r, sc in enumerate(reps):
        if len(sc["x"]) == 0:
            assert not np.any(pairs[:, 0] == r) and e[r] == 0
            continue
        xo = sc["x"] if precision else _f32(sc["x"])
        ref = oracle.forces_cells(xo, None, _op(sc), pairs=True)
        mine = pairs[pairs[:, 0] == r][:, 1:]
        assert np.array_equal(oracle.sorted_pairs(mine), oracle.sorted_pairs(ref["pairs"])), r
        if ref["count"]:
            rel = np.linalg.norm(Fr[r] - ref["F"]) / np.linalg.norm(ref["F"])
            assert rel <= force_tol, (r, rel)
            assert abs(e[r] - ref["U"]) <= (1e-12 if precision else 1e-5) * max(abs(ref["U"]), 1.0), r
            assert abs(w[r] - ref["W"]) <= (1e-12 if precision else 1e-5) * max(abs(ref["W"]), 1.0), r
        else:
            assert np.abs(Fr[r]).max() == 0 and e[r] == 0


@pytest.mark.parametrize("precision", [0, 1], ids=["fp32", "fp64"])
@pytest.mark.parametrize("tile", [(1, 128, 0), (4, 256, 0), (2, 128, 4), (8, 64, 0)])
def test_batch_pairs_forces_step0(precision, tile):
    reps = _small_batch()
    b = lj.Batch(reps, precision=precision)
    b.set_tile(threads_per_particle=tile[0], block_threads=tile[1], persistent_ctas_per_sm=tile[2])
    _check_step0(b, reps, precision, 1e-12 if precision else FORCE_TOL)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp32", "fp64"])
def test_batch_edge_replicas(precision):
    reps = _edge_batch()
    b = lj.Batch(reps, precision=precision)
    _check_step0(b, reps, precision, 1e-12 if precision else FORCE_TOL)
    b.step(25)
    x, v = b.state()
    xs = b.split(x)
    assert xs[1].shape == (0, 3)
    # the lone pair is out of range: straight-line motion
    two = reps[3]
    assert np.abs(_wrapdiff(xs[3], two["x"] + 25 * two["dt"] * two["v"], 5.7)).max() < 1e-12


def test_batch_fp64_trajectories_match_oracle():
    """FP64 batch, 60 steps (rebuilds every 10 steps and on the skin/2 rule):
    every replica's positions and velocities equal the oracle's own run."""
    reps = _small_batch(seed=44, nrep=12)
    b = lj.Batch(reps, precision=1)
    b.step(60)
    x, v = b.state()
    for r, (xr, vr, sc) in enumerate(zip(b.split(x), b.split(v), reps)):
        xo, vo, *_ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], _op(sc), sc["dt"], 60)
        assert np.abs(_wrapdiff(xr, xo, sc["box"][0])).max() < 1e-9, r
        assert np.abs(vr - vo).max() < 1e-9, r
    c = b.counters()
    assert c["steps"] == 60 and c["rebuilds"] >= 6
    # each event re-lists only the replicas that need it
    assert c["replica_rebuilds"] < len(reps) * c["rebuilds"], c


def test_batch_fp32_tracks_fp64_and_conserves_energy():
    reps = _small_batch(seed=45, nrep=8)
    b = lj.Batch(reps)
    _, e0, _ = b.compute()
    x0, v0 = b.state()
    k0 = np.array([0.5 * (vr * vr).sum() for vr in b.split(v0)])
    b.step(100)
    x, v = b.state()
    _, e1, _ = b.compute()
    k1 = np.array([0.5 * (vr * vr).sum() for vr in b.split(v)])
    for r, sc in enumerate(reps):
        tot0, tot1 = e0[r] + k0[r], e1[r] + k1[r]
        assert abs(tot1 - tot0) < 2e-3 * abs(k0[r]), (r, tot0, tot1)
        xo, *_ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], _op(sc), sc["dt"], 100)
        assert np.abs(_wrapdiff(b.split(x)[r], xo, sc["box"][0])).max() < 1e-3, r


def test_batch_graph_equals_eager():
    reps = _small_batch(seed=46, nrep=6)
    a = lj.Batch(reps)
    c = lj.Batch(reps)
    a.step(37)
    c.step(37, eager=True)
    xa, va = a.state()
    xc, vc = c.state()
    assert np.array_equal(xa, xc) and np.array_equal(va, vc)


def test_batch_equals_single_systems_fp64():
    """Each replica of an FP64 batch follows the same trajectory as the same
    system run alone through the single-system path."""
    reps = _small_batch(seed=47, nrep=4)
    b = lj.Batch(reps, precision=1)
    b.step(80)
    x, v = b.state()
    for r, sc in enumerate(reps):
        s = lj.System(sc, precision=1)
        s.step(80)
        xs, vs = s.state()
        assert np.abs(_wrapdiff(b.split(x)[r], xs, sc["box"][0])).max() < 1e-11, r
        s.close()


DEFAULT_TILES = [(t, blk, 0) for t in (1, 2, 4, 8) for blk in (128, 256)] + [(1, 128, 8), (2, 256, 4)]


def test_batch_autotune_picks_the_fastest_tile():
    reps = _small_batch(seed=48, nrep=10)
    b = lj.Batch(reps)
    chosen, costs = b.autotune(trial_steps=5)
    assert len(costs) == 10 and min(costs) > 0
    assert chosen.as_tuple()[:3] == DEFAULT_TILES[int(np.argmin(costs))]
    assert b.tile() == chosen.as_tuple()
    assert b.counters()["steps"] == 10 * 6  # every trial advances the batch (1 + 5 steps each)


def test_batch_capacity_overflow_is_recovered():
    """A dense droplet in a mostly empty box: the list capacity estimated
    from the mean densities is too small, the build reports it and the
    library grows the lists and rebuilds; results stay exact."""
    edge = _edge_batch()
    xd, _ = scenarios.fcc_lattice(4, 1.1)
    rng = np.random.default_rng(51)
    drop = dict(edge[0], x=xd + 3.0, v=rng.normal(0, 0.5, xd.shape), types=np.zeros(len(xd), np.int32),
                box=np.full(3, 24.0))
    reps = [edge[3], drop, edge[1]]
    b = lj.Batch(reps)
    _check_step0(b, reps, 0, FORCE_TOL)
    assert b.counters()["capacity_retries"] >= 1


def test_batch_full_size_sampled():
    """The full 512-replica batch (about 1.17M particles) in the tuned launch
    configuration: pair sets and forces of sampled replicas (the smallest,
    the largest, the densest and a seeded sample) against the oracle at step
    0, then 40 FP64 steps against the oracle's trajectories."""
    reps = scenarios.replica_batch()
    counts = np.array([len(r["x"]) for r in reps])
    dens = np.array([r["density"] for r in reps])
    rng = np.random.default_rng(49)
    pick = sorted(set([int(counts.argmin()), int(counts.argmax()), int(dens.argmax())] +
                      rng.choice(len(reps), 9, replace=False).tolist()))
    b = lj.Batch(reps)
    b.autotune(trial_steps=3)
    chosen = b.tile()
    # a fresh batch at step 0 in the chosen tile
    b = lj.Batch(reps)
    b.set_tile(threads_per_particle=chosen[0], block_threads=chosen[1], persistent_ctas_per_sm=chosen[2])
    F, e, w = b.compute()
    pairs = b.pairs()
    Fr = b.split(F)
    for r in pick:
        sc = reps[r]
        ref = oracle.forces_cells(_f32(sc["x"]), None, _op(sc), pairs=True)
        mine = pairs[pairs[:, 0] == r][:, 1:]
        assert np.array_equal(oracle.sorted_pairs(mine), oracle.sorted_pairs(ref["pairs"])), r
        assert np.linalg.norm(Fr[r] - ref["F"]) / np.linalg.norm(ref["F"]) <= FORCE_TOL, r
    b.close()
    b = lj.Batch(reps, precision=1)
    b.set_tile(threads_per_particle=chosen[0], block_threads=chosen[1], persistent_ctas_per_sm=chosen[2])
    b.step(40)
    x, v = b.state()
    xs = b.split(x)
    for r in pick[:6]:
        sc = reps[r]
        xo, *_ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], _op(sc), sc["dt"], 40)
        assert np.abs(_wrapdiff(xs[r], xo, sc["box"][0])).max() < 1e-9, r
