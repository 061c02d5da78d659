"""The allocation-free force entry point, through the C ABI.

ljsel_compute_forces_noalloc serves callers that cannot allocate device
memory: code inside a framework whose allocator has reserved all device
memory and forbids allocations behind its back, plug-ins running inside a
host application that owns the device, and latency-critical loops that must
not take the allocator's locks or the implicit synchronization of a free.
It keeps its intermediate arrays in one static device array of the library
(131,072 particles and 131,072 cells at most).

Checked here, each case on the GPU:
  - two calls in a row on different systems (the second smaller, with two
    particle types, so stale contents of the shared array would show)
    against ljsel_create + ljsel_compute on the same input, and against the
    FP64 oracle on the working positions (the positions wrapped into the box
    and rounded to FP32): forces within 1e-5 relative RMS, energy and
    virial within 2e-6;
  - n = 131,072 accepted and checked against the oracle; n = 131,073 and a
    box that needs more than 131,072 cells rejected with LJSEL_ERR_CAPACITY;
  - the smallest box (two cells a side) and a two-type mixture against the
    oracle;
  - repeated calls leave the device's free memory unchanged.
This file is collected last, so a run that stops at the first failure has
run every other test before it.
"""
import numpy as np
import pytest

import oracle
from paper_2505_03438_gb300 import scenarios

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
SUM_TOL = 2e-6


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_03438_gb300 as lj
    return torch, lj


def _work_positions(x, box):
    """The positions the call computes with: wrapped into [0, L) in FP64
    (x - L floor(x / L), L itself mapped to 0), then rounded to FP32."""
    L = np.broadcast_to(np.asarray(box, np.float64), (3,))
    w = x - L * np.floor(x / L)
    w = np.where(w < L, w, 0.0)
    return w.astype(np.float32).astype(np.float64)


def _jittered_mixture(seed, nside):
    """The binary mixture moved off its simple-cubic lattice by a seeded
    displacement of up to 0.08 per coordinate: on the perfect lattice
    thousands of pairs sit at one distance, so their FP32 rounding errors
    add up coherently while repulsive and attractive energies cancel, and
    the relative energy error of any FP32 pair arithmetic there is well
    above the 2e-6 bar."""
    sc = scenarios.binary_mixture(seed=seed, nside=nside)
    rng = np.random.default_rng(seed + 1000)
    sc["x"] = sc["x"] + rng.uniform(-0.08, 0.08, sc["x"].shape)
    return sc


def _noalloc(torch, lj, sc):
    p = lj.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], sc["mass"], sc["skin"], sc["dt"])
    x = torch.tensor(sc["x"], device="cuda")
    t = torch.tensor(sc["types"], dtype=torch.int32, device="cuda")
    F = torch.full_like(x, float("nan"))
    e, w = lj.ljsel_compute_forces_noalloc(p, len(sc["x"]), x, F, t)
    torch.cuda.synchronize()
    return F.cpu().numpy(), e, w


def _against_oracle(sc, F, e, w):
    op = oracle.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], sc.get("shift", True))
    ref = oracle.forces_cells(_work_positions(sc["x"], sc["box"]), sc["types"], op)
    assert np.isfinite(F).all()
    rel = np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"])
    assert rel <= FORCE_TOL, rel
    assert abs(e - ref["U"]) <= SUM_TOL * abs(ref["U"]), (e, ref["U"])
    assert abs(w - ref["W"]) <= SUM_TOL * abs(ref["W"]), (w, ref["W"])


def test_noalloc_matches_allocating_path_and_oracle(env):
    torch, lj = env
    cases = [scenarios.fcc_liquid(8, seed=81, jitter=0.15), _jittered_mixture(82, 10)]
    for sc in cases:
        Fn, e, w = _noalloc(torch, lj, sc)
        ref = lj.System(sc)
        ref.set_config(method="LC", newton3=False, csf=1.0)
        Fr, er, wr = ref.compute()
        ref.close()
        rel = np.linalg.norm(Fn - Fr) / np.linalg.norm(Fr)
        assert rel <= FORCE_TOL, rel
        assert abs(e - er) <= SUM_TOL * abs(er), (e, er)
        assert abs(w - wr) <= SUM_TOL * abs(wr), (w, wr)
        _against_oracle(sc, Fn, e, w)


def test_noalloc_limits(env):
    torch, lj = env
    # the largest accepted system: fcc 32^3 x 4 = 131,072, drifted off the lattice
    sc = scenarios.fcc_liquid(32, seed=83, jitter=0.12)
    assert len(sc["x"]) == 131072
    Fn, e, w = _noalloc(torch, lj, sc)
    _against_oracle(sc, Fn, e, w)
    # one particle more: refused before any work
    p = lj.make_params(sc["box"], skin=sc["skin"])
    x = torch.zeros((131073, 3), dtype=torch.float64, device="cuda")
    F = torch.zeros_like(x)
    with pytest.raises(lj.LjselError) as ex:
        lj.ljsel_compute_forces_noalloc(p, 131073, x, F)
    assert ex.value.status == 4
    # a dilute box of side 130: 51^3 = 132,651 cells of side >= 2.5 is over the limit
    gas = scenarios.random_gas(500, 130.0, seed=84)
    p = lj.make_params(gas["box"], skin=gas["skin"])
    x = torch.tensor(gas["x"], device="cuda")
    F = torch.zeros_like(x)
    with pytest.raises(lj.LjselError) as ex:
        lj.ljsel_compute_forces_noalloc(p, 500, x, F)
    assert ex.value.status == 4


def test_noalloc_smallest_box_and_two_types(env):
    torch, lj = env
    # L = 5.75: two cells of side >= 2.5 a side, every stencil wraps onto them
    for seed in range(5):
        sc = scenarios.random_gas(150, 5.75, seed=85 + seed, min_dist=0.8)
        Fn, e, w = _noalloc(torch, lj, sc)
        _against_oracle(sc, Fn, e, w)
    sc = _jittered_mixture(86, 7)
    Fn, e, w = _noalloc(torch, lj, sc)
    _against_oracle(sc, Fn, e, w)


def test_noalloc_repeated_calls_allocate_nothing(env):
    torch, lj = env
    sc = scenarios.fcc_liquid(6, seed=87, jitter=0.1)
    p = lj.make_params(sc["box"], skin=sc["skin"])
    x = torch.tensor(sc["x"], device="cuda")
    F = torch.zeros_like(x)
    lj.ljsel_compute_forces_noalloc(p, len(sc["x"]), x, F)  # first call: resolves the scratch address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        lj.ljsel_compute_forces_noalloc(p, len(sc["x"]), x, F)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
