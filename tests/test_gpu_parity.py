"""GPU path against the FP64 oracle, through the C ABI.

Bars: the within-cutoff pair set is bit-exact (the oracle evaluates the exact
FP64 predicate on the working positions the GPU uses); FP32 forces are within
1e-5 relative RMS of the oracle's FP64 forces on those positions; energy and
virial within 2e-6 relative (FP32 pair terms summed in FP64); the FP64 check
path matches the oracle to 1e-12.

The oracle only ever sees generator data.  The working positions of the FP32
path are the generator's positions rounded to float32 (rounded here, in
numpy).  Lists reused with drifted positions are checked by moving the
particles through ljsel_move_particles by generator-made displacements below
skin/2 (some across a box face), which keeps the lists of the last rebuild.
After simulated steps, the FP64 path is compared with the oracle's own
trajectory.
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


CONFIGS = [
    dict(method="LC", newton3=False, csf=1.0),
    dict(method="LC", newton3=True, csf=1.0),
    dict(method="LC", newton3=False, csf=0.5),
    dict(method="LC", newton3=True, csf=0.5),
    dict(method="VL", newton3=False, threads_per_unit=1),
    dict(method="VL", newton3=False, threads_per_unit=4),
    dict(method="VL", newton3=True, threads_per_unit=1),
    dict(method="VL", newton3=True, threads_per_unit=4),
    dict(method="VL", newton3=False, threads_per_unit=1, csf=0.5),
    dict(method="VL", newton3=False, threads_per_unit=2, csf=0.5),
    dict(method="VL", newton3=True, threads_per_unit=1, csf=0.5),
    dict(method="VLW", newton3=False),
    dict(method="VLW", newton3=True),
    dict(method="CL", cluster_size=2, newton3=False, threads_per_unit=2),
    dict(method="CL", cluster_size=2, newton3=False, threads_per_unit=8),
    dict(method="CL", cluster_size=2, newton3=True, threads_per_unit=4),
    dict(method="CL", cluster_size=4, newton3=False, threads_per_unit=4),
    dict(method="CL", cluster_size=4, newton3=False, threads_per_unit=16),
    dict(method="CL", cluster_size=4, newton3=True, threads_per_unit=8),
    dict(method="CL", cluster_size=8, newton3=False, threads_per_unit=8),
    dict(method="CL", cluster_size=8, newton3=False, threads_per_unit=32),
    dict(method="CL", cluster_size=8, newton3=True, threads_per_unit=8),
    dict(method="CL", cluster_size=4, newton3=False, threads_per_unit=8, csf=0.5),
    dict(method="CL", cluster_size=4, newton3=True, threads_per_unit=4, csf=0.5),
]


def cfg_id(c):
    return "%s%s-%s-t%d-csf%g" % (c["method"], c.get("cluster_size", ""), "n3" if c["newton3"] else "full",
                                 c.get("threads_per_unit", 1), c.get("csf", 1.0))


def _systems():
    out = {
        "jfcc864": scenarios.fcc_liquid(6, seed=11, jitter=0.15),
        "gas500": scenarios.random_gas(500, 12.0, seed=12, min_dist=0.8),
        "tinybox": scenarios.random_gas(150, 5.75, seed=13, min_dist=0.8),
        "binary": scenarios.binary_mixture(seed=14, nside=12),
    }
    return out


SYSTEMS = _systems()


def _orc_params(sc):
    return oracle.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], sc.get("shift", True))


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def drift(x, box, seed, amp):
    """Generator-made displacement of every particle by less than amp, with
    particles next to a box face stepping across it (positions stay
    unwrapped, as between rebuilds)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=x.shape)
    d *= (amp * rng.uniform(0.2, 1.0, (len(x), 1))) / np.linalg.norm(d, axis=1, keepdims=True)
    L = np.broadcast_to(np.asarray(box, np.float64), (3,))
    d = np.where(x < 0.5 * amp, -np.abs(d), d)
    d = np.where(x > L - 0.5 * amp, np.abs(d), d)
    return x + d


def check_against_oracle(sys_, sc, x, precision=0, force_tol=FORCE_TOL, sum_tol=SUM_TOL, forces=True):
    """Forces, energy, virial and pair set of the system, whose positions are
    x (generator data), against the oracle on the working positions.  On a
    perfect lattice every force cancels to rounding, so there the relative
    force error is not defined and forces=False skips it."""
    F, e, w = sys_.compute()
    xw = x if precision else _f32(x)
    ref = oracle.forces_cells(xw, sc["types"], _orc_params(sc), pairs=True)
    pairs, cnt = sys_.pairs()
    assert cnt == ref["count"], (cnt, ref["count"])
    assert np.array_equal(oracle.sorted_pairs(pairs), oracle.sorted_pairs(ref["pairs"]))
    rel = np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"]) if forces else 0.0
    assert rel <= force_tol, rel
    assert abs(e - ref["U"]) <= sum_tol * max(abs(ref["U"]), 1.0), (e, ref["U"])
    assert abs(w - ref["W"]) <= sum_tol * max(abs(ref["W"]), 1.0), (w, ref["W"])
    return rel


@pytest.mark.parametrize("cfg", CONFIGS, ids=cfg_id)
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_pairs_forces_fp32(lj, cfg, name):
    sc = SYSTEMS[name]
    s = lj.System(sc)
    s.set_config(rebuild_interval=10, **cfg)
    check_against_oracle(s, sc, sc["x"])
    # drifted (not wrapped) positions with the lists of the last rebuild
    nreb = s.counters()["rebuilds"]
    x1 = drift(sc["x"], sc["box"], 1000 + len(sc["x"]), 0.9 * 0.5 * sc["skin"])
    s.move_particles(x1)
    check_against_oracle(s, sc, x1)
    assert s.counters()["rebuilds"] == nreb
    s.close()


@pytest.mark.parametrize("cfg", CONFIGS, ids=cfg_id)
def test_pairs_forces_fp64(lj, cfg):
    for name in ("jfcc864", "binary"):
        sc = SYSTEMS[name]
        s = lj.System(sc, precision=1)
        s.set_config(rebuild_interval=10, **cfg)
        check_against_oracle(s, sc, sc["x"], 1, force_tol=1e-12, sum_tol=1e-12)
        x1 = drift(sc["x"], sc["box"], 2000 + len(sc["x"]), 0.9 * 0.5 * sc["skin"])
        s.move_particles(x1)
        check_against_oracle(s, sc, x1, 1, force_tol=1e-12, sum_tol=1e-12)
        # past skin/2 the next evaluation rebuilds first
        x2 = drift(sc["x"], sc["box"], 3000 + len(sc["x"]), 2.0 * sc["skin"])
        nreb = s.counters()["rebuilds"]
        s.move_particles(x2)
        check_against_oracle(s, sc, x2, 1, force_tol=1e-12, sum_tol=1e-12)
        assert s.counters()["rebuilds"] >= nreb + 1  # (one more if the longer rows overflow the fitted capacity)
        s.close()


def _wrapdiff(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def test_fp64_trajectory_small_fcc(lj):
    """Plain method in FP64: N = 4000 fcc, linked cells of side >= r_c, 100 NVE
    steps; the GPU trajectory equals the oracle's up to rounding."""
    sc = scenarios.small_fcc()
    s = lj.System(sc, precision=1)
    s.set_config(method="LC", newton3=False, rebuild_interval=1, csf=1.0)
    ep0, ek0, _ = s.energy()
    s.step(sc["nsteps"])
    x, v = s.state()
    ep1, ek1, _ = s.energy()
    xo, vo, epo, eko, _ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], _orc_params(sc), sc["dt"], sc["nsteps"])
    L = sc["box"][0]
    assert np.abs(_wrapdiff(x, xo, L)).max() < 1e-10
    assert np.abs(v - vo).max() < 1e-10
    assert abs(ep0 - epo[0]) < 1e-10 * abs(epo[0]) and abs(ek0 - eko[0]) < 1e-10 * abs(eko[0])
    assert abs(ep1 - epo[-1]) < 1e-9 * abs(epo[-1]) and abs(ek1 - eko[-1]) < 1e-9 * abs(eko[-1])
    s.close()


@pytest.mark.parametrize("method", ["VL", "LC", "CL", "VLW"])
def test_fp32_trajectory_tracks_fp64(lj, method):
    sc = scenarios.fcc_liquid(8, seed=21, jitter=0.05)
    s = lj.System(sc)
    kw = dict(method=method, rebuild_interval=10)
    if method == "CL":
        kw.update(cluster_size=8, threads_per_unit=8)
    s.set_config(**kw)
    e0 = sum(s.energy()[:2])
    s.step(100)
    x, v = s.state()
    e1 = sum(s.energy()[:2])
    xo, vo, epo, eko, _ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], _orc_params(sc), sc["dt"], 100)
    L = sc["box"][0]
    assert abs(e1 - e0) < 1e-3 * abs(e0)
    assert abs(e1 - (epo[-1] + eko[-1])) < 1e-4 * abs(e0)
    assert np.abs(_wrapdiff(x, xo, L)).max() < 1e-3
    s.close()


def test_graph_equals_eager(lj):
    sc = scenarios.fcc_liquid(6, seed=31, jitter=0.1)
    out = []
    for g in (True, False):
        s = lj.System(sc, use_graphs=g)
        s.set_config(method="VL", rebuild_interval=7)
        s.step(45)
        out.append(s.state())
        c = s.counters()
        assert c["steps"] == 45
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("cfg", [dict(method="VL"), dict(method="VL", csf=0.5), dict(method="VL", newton3=True, csf=0.5)],
                         ids=["csf1", "csf0.5", "n3-csf0.5"])
def test_displacement_forces_early_rebuild(lj, cfg):
    # hot gas: particles cross skin/2 long before R = 200 steps; the FP64 run
    # stays on the oracle's trajectory, so no pair was missed
    sc = scenarios.random_gas(800, 14.0, seed=41, min_dist=0.9, temperature=6.0)
    s = lj.System(sc, skin=0.2, precision=1)
    s.set_config(rebuild_interval=200, **cfg)
    s.step(120)
    c = s.counters()
    assert c["early_rebuilds"] >= 2, c
    x, v = s.state()
    xo, vo, *_ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], _orc_params(sc), sc["dt"], 120)
    assert np.abs(_wrapdiff(x, xo, sc["box"][0])).max() < 1e-9
    assert np.abs(v - vo).max() < 1e-9
    pairs, cnt = s.pairs()
    ref = oracle.forces_cells(xo, None, _orc_params(sc), pairs=True)
    assert np.array_equal(oracle.sorted_pairs(pairs), oracle.sorted_pairs(ref["pairs"]))
    s.close()


def test_capacity_overflow_is_recovered(lj):
    # a dense droplet in a large sparse box: the mean-density estimate of the
    # list length is far too small, the first build overflows and is redone
    rng = np.random.default_rng(5)
    core = scenarios.fcc_lattice(5, 0.9)[0]
    core = core - core.mean(0) + 15.0
    gas = rng.uniform(0, 30.0, (300, 3))
    x = np.concatenate([core, gas])
    keep = np.ones(len(x), bool)
    for k in range(len(core), len(x)):
        d = np.abs(x[:k][keep[:k]] - x[k])
        d = np.minimum(d, 30.0 - d)
        if ((d * d).sum(1) < 0.81).any():
            keep[k] = False
    x = x[keep]
    v = scenarios.maxwell_boltzmann(len(x), 1.0, 1.0, rng)
    sc = dict(x=x, v=v, types=np.zeros(len(x), np.int32), box=np.full(3, 30.0), eps=np.ones((1, 1)),
              sigma=np.ones((1, 1)), rcut=np.full((1, 1), 2.5), mass=np.ones(1), skin=0.3, dt=0.005, shift=True)
    for cfg in (dict(method="VL"), dict(method="CL", cluster_size=8, threads_per_unit=8)):
        s = lj.System(sc)
        s.set_config(**cfg)
        check_against_oracle(s, sc, x)
        if cfg["method"] == "VL":
            assert s.counters()["capacity_retries"] >= 1
        x1 = drift(x, sc["box"], 77, 0.13)
        s.move_particles(x1)
        check_against_oracle(s, sc, x1)
        s.close()


def test_live_statistics(lj):
    for sc in (scenarios.fcc_liquid(7, seed=51, jitter=0.2), scenarios.random_gas(400, 14.0, seed=52, min_dist=0.8)):
        s = lj.System(sc)
        s.step(10)
        st = s.stats()
        x, _ = s.state()
        ref = oracle.bin_stats(x, sc["box"], 2.5 + sc["skin"])
        for k in ("mean", "rel_std", "median", "max", "nbins", "nempty"):
            assert abs(st[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (k, st[k], ref[k])
        # the thread count: the device's resident threads, whatever the configuration
        import torch
        props = torch.cuda.get_device_properties(0)
        assert st["threads"] == props.multi_processor_count * props.max_threads_per_multi_processor
        assert st["skin"] == sc["skin"]
        s.set_config(method="VL", threads_per_unit=4)
        assert s.stats()["threads"] == st["threads"]
        s.close()


def _on_oracle_trajectory(s, sc):
    """An FP64 system whose trial steps switched configuration mid-run is
    still on the oracle's trajectory."""
    nsteps = s.counters()["steps"]
    x, v = s.state()
    xo, vo, *_ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], _orc_params(sc), sc["dt"], nsteps)
    assert np.abs(_wrapdiff(x, xo, sc["box"][0])).max() < 1e-8, nsteps
    assert np.abs(v - vo).max() < 1e-8, nsteps


def test_autotune_full_and_predictive(lj):
    sc = scenarios.fcc_liquid(8, seed=61, jitter=0.1)
    s = lj.System(sc, precision=1)
    cands = lj.ljsel_default_candidates(s.h)
    assert len(cands) >= 15
    chosen, rep = s.autotune(strategy=0, trial_steps=10)
    assert rep["ntrialled"] == len(cands) and rep["chosen_cost_ms"] > 0
    assert any(chosen.name() == c.name() for c in cands)
    assert s.config().name() == chosen.name()
    assert s.counters()["steps"] == 10 * len(cands)
    _on_oracle_trajectory(s, sc)
    # predictive strategy: two full phases, then a filtered one
    s2 = lj.System(sc, precision=1)
    for ph in range(3):
        _, rep = s2.autotune(strategy=1, trial_steps=10, blacklist_factor=10.0)
    assert rep["ntrialled"] < len(cands)
    _on_oracle_trajectory(s2, sc)
    # probe filter: slow configurations stop after their probe steps
    s3 = lj.System(sc, precision=1)
    _, rep = s3.autotune(strategy=0, trial_steps=10, probe_steps=2, probe_factor=1.5)
    assert rep["nprobed_out"] > 0 and rep["trial_steps_total"] < 10 * len(cands)
    assert s3.counters()["steps"] == rep["trial_steps_total"]
    _on_oracle_trajectory(s3, sc)
    # expert strategy: the dense liquid (about 16 particles per bin) trials
    # the Verlet and cluster lists only
    s4 = lj.System(sc)
    chosen4, rep = s4.autotune(strategy="expert", trial_steps=5)
    assert rep["expert_input"] > 8
    assert rep["ntrialled"] == sum(c.method in (lj.METHOD_VL, lj.METHOD_CLUSTER) for c in cands)
    assert chosen4.method in (lj.METHOD_VL, lj.METHOD_CLUSTER)
    # the FP32 system keeps the selected configuration's exactness: moved
    # particles with its lists against the oracle
    x1 = drift(sc["x"], sc["box"], 62, 0.05)
    s4.set_state(sc["x"], sc["v"])
    check_against_oracle(s4, sc, sc["x"])
    s4.move_particles(x1)
    check_against_oracle(s4, sc, x1)
    for x in (s, s2, s3, s4):
        x.close()


def test_device_pointer_inputs(lj):
    import torch
    sc = scenarios.fcc_liquid(5, seed=71, jitter=0.1)
    x = torch.tensor(sc["x"], device="cuda")
    v = torch.tensor(sc["v"], device="cuda")
    t = torch.zeros(len(sc["x"]), dtype=torch.int32, device="cuda")
    p = lj.make_params(sc["box"], skin=0.3)
    h = lj.ljsel_create(p, len(sc["x"]), x, v, t, torch.cuda.current_stream().cuda_stream)
    F = torch.zeros_like(x)
    e, w = lj.ljsel_compute(h, F)
    torch.cuda.synchronize()
    ref = oracle.forces_cells(_f32(sc["x"]), None, _orc_params(sc))
    Fh = F.cpu().numpy()
    assert np.linalg.norm(Fh - ref["F"]) / np.linalg.norm(ref["F"]) < FORCE_TOL
    lj.ljsel_destroy(h)


def test_liquid_1m_full_size(lj):
    """Full-size homogeneous liquid (N = 1,048,576) in the benchmark's launch
    configuration: whole pair set and all forces against the oracle."""
    sc = scenarios.liquid_1m()
    x1 = drift(sc["x"], sc["box"], 81, 0.9 * 0.5 * sc["skin"])
    for cfg in (dict(method="VL"), dict(method="VL", csf=0.5), dict(method="VL", newton3=True, csf=0.5),
                dict(method="VLW"), dict(method="VLW", newton3=True)):
        s = lj.System(sc)
        s.set_config(rebuild_interval=10, **cfg)
        check_against_oracle(s, sc, sc["x"], forces=False)  # perfect fcc lattice: all forces vanish
        s.move_particles(x1)
        check_against_oracle(s, sc, x1)
        s.close()


SMALL_BOX_CFGS = [dict(method="VL"), dict(method="VL", newton3=True), dict(method="VL", csf=0.5),
                  dict(method="VL", newton3=True, csf=0.5), dict(method="LC"), dict(method="LC", csf=0.5),
                  dict(method="CL", cluster_size=4, threads_per_unit=4),
                  dict(method="CL", cluster_size=2, newton3=True, threads_per_unit=2),
                  dict(method="CL", cluster_size=8, newton3=True, threads_per_unit=8, csf=0.5), dict(method="VLW")]


@pytest.mark.parametrize("cfg", SMALL_BOX_CFGS, ids=lambda c: "-".join("%s%s" % kv for kv in c.items()))
def test_smallest_boxes_twenty_seeds(lj, cfg):
    """The smallest box the library accepts (L = 2 (r_c + skin)(1 + 2^-10),
    plus 0.01): two cells per side (four at CSF 0.5), every stencil wraps
    onto the same cells with two images; 20 seeded random gases, pair sets
    and forces exact."""
    L = 2 * 2.8 * (1 + 1.0 / 1024) + 0.01
    kw = dict(cfg, rebuild_interval=10)
    for seed in range(20):
        sc = scenarios.random_gas(120, L, seed=100 + seed, min_dist=0.8)
        s = lj.System(sc)
        s.set_config(**kw)
        check_against_oracle(s, sc, sc["x"])
        s.close()


@pytest.mark.parametrize("n3l_cfg", [dict(method="VL", newton3=True), dict(method="LC", newton3=True),
                                     dict(method="CL", cluster_size=4, newton3=True, threads_per_unit=4)],
                         ids=["VL", "LC", "CL4"])
def test_switch_to_newton3_after_a_force_evaluation(lj, n3l_cfg):
    """A force evaluation without N3L leaves its forces in the buffer that N3L
    kernels accumulate into; switching to an N3L configuration must not
    carry them into the next steps (FP64 path on the oracle's trajectory)."""
    sc = scenarios.fcc_liquid(5, seed=17, jitter=0.1)
    s = lj.System(sc, precision=1)
    s.compute()
    s.set_config(rebuild_interval=10, **n3l_cfg)
    s.step(10)
    x, v = s.state()
    xo, vo, *_ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], _orc_params(sc), sc["dt"], 10)
    assert np.abs(_wrapdiff(x, xo, sc["box"][0])).max() < 1e-10
    assert np.abs(v - vo).max() < 1e-10


def test_unshifted_potential_and_unequal_masses_fp64(lj):
    """Energy without the shift at r_c, and a binary mixture whose species
    have masses 1 and 2: the FP64 trajectory is the oracle's."""
    sc = dict(scenarios.binary_mixture(seed=15, nside=9), shift=False, mass=np.array([1.0, 2.0]))
    p = oracle.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], False)
    s = lj.System(sc, precision=1)
    F, e, w = s.compute()
    ref = oracle.forces_cells(sc["x"], sc["types"], p)
    assert np.abs(F - ref["F"]).max() < 1e-11 * np.abs(ref["F"]).max()
    assert abs(e - ref["U"]) < 1e-11 * abs(ref["U"]) and abs(w - ref["W"]) < 1e-11 * abs(ref["W"])
    s.step(40)
    x, v = s.state()
    xo, vo, epo, eko, _ = oracle.verlet_run(sc["x"], sc["v"], sc["types"], sc["mass"], p, sc["dt"], 40)
    assert np.abs(_wrapdiff(x, xo, sc["box"][0])).max() < 1e-10
    assert np.abs(v - vo).max() < 1e-10
    ep, ek, _ = s.energy()
    assert abs(ep - epo[-1]) < 1e-9 * abs(epo[-1]) and abs(ek - eko[-1]) < 1e-9 * abs(eko[-1])


ROW_CFGS = [dict(method="VL"), dict(method="VL", newton3=True), dict(method="VL", csf=0.5),
            dict(method="VL", threads_per_unit=4), dict(method="VLW"), dict(method="VLW", newton3=True),
            dict(method="CL", cluster_size=4, threads_per_unit=4),
            dict(method="CL", cluster_size=2, newton3=True, threads_per_unit=2)]


@pytest.mark.parametrize("cfg", ROW_CFGS, ids=lambda c: "-".join("%s%s" % kv for kv in c.items()))
def test_rows_ending_at_their_capacity(lj, cfg):
    """List rows that end exactly at their capacity or within one 16-byte
    chunk of it, with periodic-image entries at the back of the row: in a box
    just above the smallest accepted one most rows carry image entries.  The
    row capacity is set to the longest row of the build (rounded up to the
    row granularity) and to one chunk more; the structure must be built
    without growing the rows, and pair sets and forces must match the oracle
    at the build positions and after a drift that keeps the lists."""
    L = 2 * 2.8 * (1 + 1.0 / 1024) + 0.3
    unit = 16 if cfg["method"] == "VLW" else 4
    for seed in range(4):
        sc = scenarios.random_gas(170, L, seed=300 + seed, min_dist=0.8)
        s = lj.System(sc)
        s.set_config(rebuild_interval=10, **cfg)
        s.compute()
        longest = s.counters()["longest_row"]
        assert longest > 0
        for cap in ((longest + unit - 1) // unit * unit, (longest + unit - 1) // unit * unit + unit):
            s.set_state(sc["x"], sc["v"])
            lj.ljsel_set_list_capacity(s.h, cap)
            retries = s.counters()["capacity_retries"]
            check_against_oracle(s, sc, sc["x"])
            c = s.counters()
            assert c["capacity_retries"] == retries and c["longest_row"] <= cap, (cap, c)
            x1 = drift(sc["x"], sc["box"], 400 + seed, 0.9 * 0.5 * sc["skin"])
            s.move_particles(x1)
            check_against_oracle(s, sc, x1)
        s.close()


def test_batch_rows_ending_at_their_capacity(lj):
    """The same for the batched replicas' rows: small boxes (about two cells
    a side), capacity set to the longest row and to one chunk more."""
    reps = [scenarios.random_gas(150, 5.7 + 0.05 * k, seed=320 + k, min_dist=0.8) for k in range(6)]
    b = lj.Batch(reps)
    b.compute()
    longest = b.counters()["longest_row"]
    assert longest > 0
    for cap in ((longest + 3) // 4 * 4, (longest + 3) // 4 * 4 + 4):
        lj.ljsel_batch_set_list_capacity(b.h, cap)
        retries = b.counters()["capacity_retries"]
        F, e, w = b.compute()
        pairs = b.pairs()
        Fr = b.split(F)
        for r, sc in enumerate(reps):
            ref = oracle.forces_cells(_f32(sc["x"]), None, _orc_params(sc), pairs=True)
            mine = pairs[pairs[:, 0] == r][:, 1:]
            assert np.array_equal(oracle.sorted_pairs(mine), oracle.sorted_pairs(ref["pairs"])), (cap, r)
            assert np.linalg.norm(Fr[r] - ref["F"]) / np.linalg.norm(ref["F"]) <= FORCE_TOL
        c = b.counters()
        assert c["capacity_retries"] == retries and c["longest_row"] <= cap, (cap, c)
    b.close()
