"""The force arithmetic of the stepping kernels against the FP64 oracle
(Sec. 2.1 forces over the traversals of Sec. 2.2.1; Sec. 2.1 Stormer-Verlet).

`ljsel_step` runs kernels that accumulate no energy or virial; for a single
particle type some of them are separate kernels with their own arithmetic
(the packed FP32x2 cluster kernel).  `System.forces()` (ljsel_compute with
both sums NULL) returns the forces of exactly those kernels, and one
`step(1)` runs the fused force + update.  Bars:
- forces: 1e-5 relative RMS, and per particle |dF_i| <= 1e-5 S_i + 1e-6 with
  S_i = sum_j |F_ij| over the oracle's pairs of i (the FP32 rounding of a
  sum of pair terms is bounded by a few ulps of S_i; a pair missed at the
  cutoff changes F_i by |F(r_c)| = 0.0156 for the 1M liquid, far above
  that);
- one step from (x0, v0): x1 = x0 + dt v0 + dt^2/2 F0/m per particle to
  1e-9 plus dt^2/2 times the force bar over m, and
  v1 - v0 = dt/2 (F0 + F1)/m within 1e-5 relative RMS, F0 and F1 the
  oracle's forces at the working positions the GPU used.
"""
import numpy as np
import pytest

import oracle
from paper_2505_03438_gb300 import scenarios
from test_gpu_parity import CONFIGS, SYSTEMS, cfg_id, drift, _orc_params, _f32

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5


@pytest.fixture(scope="module")
def lj():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_03438_gb300 as m
    return m


def pair_force_scale(x, types, sc, pairs):
    """S_i = sum over the listed pairs of i of |F_ij| (a tolerance scale)."""
    x = np.asarray(x, np.float64)
    n = len(x)
    t = np.zeros(n, np.int64) if types is None else np.asarray(types, np.int64)
    eps = np.asarray(sc["eps"], np.float64).reshape(len(sc["mass"]), -1)
    sig = np.asarray(sc["sigma"], np.float64).reshape(eps.shape)
    L = np.broadcast_to(np.asarray(sc["box"], np.float64), (3,))
    p = np.asarray(pairs, np.int64).reshape(-1, 2)
    S = np.zeros(n)
    for lo in range(0, len(p), 1 << 22):
        q = p[lo:lo + (1 << 22)]
        d = x[q[:, 0]] - x[q[:, 1]]
        d -= L * np.round(d / L)
        r2 = (d * d).sum(1)
        e = eps[t[q[:, 0]], t[q[:, 1]]]
        s2 = sig[t[q[:, 0]], t[q[:, 1]]] ** 2 / r2
        s6 = s2 * s2 * s2
        f = np.abs(24.0 * e * s6 * (2.0 * s6 - 1.0)) / np.sqrt(r2)
        S += np.bincount(q[:, 0], f, minlength=n) + np.bincount(q[:, 1], f, minlength=n)
    return S


def check_forces(F, ref, S, tag=""):
    rel = np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"])
    assert rel <= FORCE_TOL, (tag, rel)
    dev = np.linalg.norm(F - ref["F"], axis=1)
    bound = 1e-5 * S + 1e-6
    worst = int(np.argmax(dev / bound))
    assert dev[worst] <= bound[worst], (tag, worst, dev[worst], S[worst])
    return rel


@pytest.mark.parametrize("cfg", CONFIGS, ids=cfg_id)
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_stepping_forces_fp32(lj, cfg, name):
    sc = SYSTEMS[name]
    s = lj.System(sc)
    s.set_config(rebuild_interval=10, **cfg)
    p = _orc_params(sc)
    for k, x in enumerate([sc["x"], drift(sc["x"], sc["box"], 2000 + len(sc["x"]), 0.9 * 0.5 * sc["skin"])]):
        if k:
            s.move_particles(x)  # the lists of the last rebuild, positions unwrapped
        xw = _f32(x)
        ref = oracle.forces_cells(xw, sc.get("types"), p, pairs=True)
        S = pair_force_scale(xw, sc.get("types"), sc, ref["pairs"])
        if np.linalg.norm(ref["F"]) > 0:
            check_forces(s.forces(), ref, S, (name, k))
    s.close()


def _one_step_check(s, sc, x0, v0, p):
    """One ljsel_step from (x0, v0) against the velocity-form Verlet step
    with the oracle's forces at the working positions the GPU used."""
    dt = sc["dt"]
    m = np.asarray(sc["mass"], np.float64)[np.zeros(len(x0), np.int64) if sc.get("types") is None
                                            else np.asarray(sc["types"], np.int64)][:, None]
    s.set_state(x0, v0)
    s.forces()  # the rebuild that set_state requested wraps the positions: read them after it
    w0 = s.work_positions()
    s.step(1)
    w1 = s.work_positions()
    x1, v1 = s.state()
    r0 = oracle.forces_cells(w0, sc.get("types"), p, pairs=True)
    F0 = r0["F"]
    S0 = pair_force_scale(w0, sc.get("types"), sc, r0["pairs"])
    del r0
    F1 = oracle.forces_cells(w1, sc.get("types"), p)["F"]
    L = np.broadcast_to(np.asarray(sc["box"], np.float64), (3,))
    xe = x0 + dt * v0 + 0.5 * dt * dt * F0 / m
    dxw = np.linalg.norm(x1 - xe - L * np.round((x1 - xe) / L), axis=1)
    # the FP32 force enters x1 through dt^2/2 F0 / m: the force bar per particle
    xtol = 1e-9 + 0.5 * dt * dt * (1e-5 * S0 + 1e-6) / m[:, 0]
    worst = int(np.argmax(dxw / xtol))
    assert dxw[worst] <= xtol[worst], (worst, dxw[worst], xtol[worst])
    dv = v1 - v0
    dv_ref = 0.5 * dt * (F0 + F1) / m
    rel = np.linalg.norm(dv - dv_ref) / np.linalg.norm(dv_ref)
    assert rel <= FORCE_TOL, rel
    return rel


@pytest.mark.parametrize("cfg", CONFIGS, ids=cfg_id)
@pytest.mark.parametrize("name", ["jfcc864", "gas500", "tinybox", "binary"])
def test_one_step_fp32(lj, cfg, name):
    sc = SYSTEMS[name]
    x0 = drift(sc["x"], sc["box"], 3000 + len(sc["x"]), 0.05)
    s = lj.System(sc)
    s.set_config(rebuild_interval=10, **cfg)
    _one_step_check(s, sc, x0, sc["v"], _orc_params(sc))
    s.close()


def test_every_candidate_liquid_1m_stepping(lj):
    """Every default candidate at N = 1,048,576: the stepping kernels'
    forces at drifted positions with the lattice's structure, then one step."""
    sc = scenarios.liquid_1m()
    x1 = drift(sc["x"], sc["box"], 92, 0.9 * 0.5 * sc["skin"])
    p = oracle.make_params(sc["box"], 1.0, 1.0, 2.5, True)
    ref = oracle.forces_cells(_f32(x1), None, p, pairs=True)
    S = pair_force_scale(_f32(x1), None, sc, ref["pairs"])
    del ref["pairs"]
    s = lj.System(sc)
    cands = lj.ljsel_default_candidates(s.h)
    for c in cands:
        s.set_state(sc["x"], sc["v"])
        lj.ljsel_set_config(s.h, c)
        s.forces()  # builds this configuration's structure at the lattice positions
        nreb = s.counters()["rebuilds"]
        s.move_particles(x1)
        check_forces(s.forces(), ref, S, c.name())
        assert s.counters()["rebuilds"] == nreb, c.name()
        _one_step_check(s, sc, x1, sc["v"], p)
    s.close()


@pytest.mark.parametrize("cfg", [dict(method="VL", threads_per_unit=2), dict(method="VL", newton3=True, threads_per_unit=4),
                                 dict(method="CL", cluster_size=4, threads_per_unit=4)], ids=["VL", "VL-N3L", "CL4"])
def test_working_positions_are_the_fp32_rounding(lj, cfg):
    """After steps the working positions (written by the update) are the
    FP32 round-to-nearest-even of the FP64 positions, bit for bit."""
    sc = scenarios.liquid_1m()
    s = lj.System(sc)
    s.set_config(rebuild_interval=10, **cfg)
    s.step(7)
    w = s.work_positions()
    x, _ = s.state()  # wrapped into [0, L); the working copy is unwrapped since the last rebuild
    L = np.broadcast_to(np.asarray(sc["box"], np.float64), (3,))
    # away from the faces no particle crossed one in 7 steps (it would have
    # to move 0.5): there the rounding must hold bit for bit
    interior = np.minimum(x, L - x) > 0.5
    x32 = np.asarray(x, np.float32).astype(np.float64)
    assert interior.mean() > 0.97
    bad = interior & (x32 != w)
    assert not bad.any(), (np.argwhere(bad)[:5], x[bad][:5], w[bad][:5])
    # near a face a coordinate that crossed it since the last rebuild is
    # exported wrapped (x - L or x + L rounded in FP64, up to 1.4e-14 off),
    # so the unwrapped value is recovered to within one FP32 ulp only
    best = np.full(x.shape, np.inf)
    for k in (-1.0, 0.0, 1.0):
        best = np.minimum(best, np.abs(np.asarray(x + k * L, np.float32).astype(np.float64) - w))
    ulp = np.spacing(np.abs(w).astype(np.float32)).astype(np.float64)
    edge = ~interior
    assert (best[edge] <= ulp[edge]).all()
    assert (best[edge] > 0).sum() <= 10
    s.close()
