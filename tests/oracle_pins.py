"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each pin takes a loaded oracle library (the real one, or a deliberately
broken build in the mutation test) and raises AssertionError when the fact
fails.  The facts:
  * closed forms of the LJ pair: U(2^(1/6) sigma) = -eps, F = 0 there,
    U(sigma) = 0, the eps/sigma scaling law, force = -dU/dr;
  * two-body direction: repulsive inside the minimum, attractive outside;
  * perfect fcc lattice: every force is zero by symmetry, the pair count is a
    shell count (12 + 6 + 24 + 12 neighbours inside 2.5 sigma), and U/N is
    the lattice sum over independently enumerated lattice vectors;
  * Newton's third law, virial = -dU/dlambda under uniform scaling;
  * two traversals (brute force and linked cells) and scipy's k-d tree give
    the same pair set;
  * NVE energy conservation with dt^2 scaling, momentum conservation and time
    reversibility of Stormer-Verlet.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle
from paper_2505_03438_gb300 import scenarios


def _p(box, rc=2.5, shift=True, eps=1.0, sigma=1.0):
    return oracle.make_params(box, eps, sigma, rc, shift)


def pin_lj_minimum(lib):
    for eps, sig in [(1.0, 1.0), (1.5, 0.8), (0.5, 0.88), (2.0, 1.3)]:
        r = 2.0 ** (1.0 / 6.0) * sig
        f, u = oracle.lj_pair(r, eps, sig, 2.5 * sig, shift=False, lib=lib)
        assert abs(f * r) < 1e-12 * eps / sig, (eps, sig, f)
        assert abs(u + eps) < 1e-13 * eps, (eps, sig, u)
        f, u = oracle.lj_pair(sig, eps, sig, 2.5 * sig, shift=False, lib=lib)
        assert abs(u) < 1e-13 * eps, (eps, sig, u)


def pin_lj_shift(lib):
    # shifted energy is continuous at r_c: U_s(r_c - h) ~ F(r_c) h -> 0
    for eps, sig, rc in [(1.0, 1.0, 2.5), (1.5, 0.8, 2.0), (0.5, 0.88, 2.2)]:
        h = 1e-7
        f_rc, _ = oracle.lj_pair(rc, eps, sig, rc, True, lib=lib)
        _, u_in = oracle.lj_pair(rc - h, eps, sig, rc, True, lib=lib)
        assert abs(u_in - f_rc * rc * h) < 1e-12, (eps, sig, u_in)
        # the shift is the unshifted energy at the cutoff
        _, u_s = oracle.lj_pair(1.3 * sig, eps, sig, rc, True, lib=lib)
        _, u_u = oracle.lj_pair(1.3 * sig, eps, sig, rc, False, lib=lib)
        _, u_c = oracle.lj_pair(rc, eps, sig, rc, False, lib=lib)
        assert abs((u_u - u_s) - u_c) < 1e-14
        assert u_c < 0


def pin_lj_scaling_and_gradient(lib):
    for eps, sig in [(1.0, 1.0), (1.5, 0.8), (0.5, 0.88)]:
        for r in np.linspace(0.9 * sig, 2.5 * sig, 23):
            f, u = oracle.lj_pair(r, eps, sig, 2.5 * sig, False, lib=lib)
            f1, u1 = oracle.lj_pair(r / sig, 1.0, 1.0, 2.5, False, lib=lib)
            assert abs(u - eps * u1) <= 1e-12 * (abs(u) + 1e-12), (eps, sig, r)
            h = 1e-6 * r
            _, up = oracle.lj_pair(r + h, eps, sig, 2.5 * sig, False, lib=lib)
            _, um = oracle.lj_pair(r - h, eps, sig, 2.5 * sig, False, lib=lib)
            dudr = (up - um) / (2 * h)
            # force magnitude along r_ij is -dU/dr = f_over_r * r
            assert abs(f * r + dudr) <= 1e-6 * (abs(dudr) + 1e-3), (eps, sig, r, f * r, dudr)


def pin_two_body(lib):
    box = np.full(3, 20.0)
    p = _p(box)
    for r, repulsive in [(1.0, True), (1.05, True), (1.2, False), (2.0, False)]:
        x = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
        out = oracle.forces_brute(x, None, p, lib=lib)
        F = out["F"]
        assert np.allclose(F[0], -F[1], rtol=0, atol=1e-14)
        assert abs(F[0, 1]) < 1e-15 and abs(F[0, 2]) < 1e-15
        # particle 0 sits at lower x: repulsion pushes it towards -x
        assert (F[0, 0] < 0) == repulsive, (r, F[0])
        # across the periodic boundary the same pair gives the same force
        xw = np.array([[0.5 * r, 5.0, 5.0], [20.0 - 0.5 * r, 5.0, 5.0]])
        Fw = oracle.forces_brute(xw, None, p, lib=lib)["F"]
        assert abs(abs(Fw[0, 0]) - abs(F[0, 0])) <= 1e-12 * abs(F[0, 0])
        assert (Fw[0, 0] > 0) == repulsive
        for cells in (False, True):
            o = oracle.forces_cells(x, None, p, lib=lib) if cells else out
            assert o["count"] == 1


def _fcc_shell_vectors(a, rc):
    """All fcc lattice vectors (conventional cube side a) shorter than rc."""
    m = int(np.ceil(rc / a)) + 1
    vecs = []
    for i, j, k in itertools.product(range(-m, m + 1), repeat=3):
        for b in scenarios.FCC_BASIS:
            v = (np.array([i, j, k]) + b) * a
            r = np.linalg.norm(v)
            if 0 < r < rc:
                vecs.append(r)
    return np.array(vecs)


def pin_fcc_lattice(lib):
    sc = scenarios.fcc_liquid(10, seed=1)
    x, box = sc["x"], sc["box"]
    p = _p(box)
    a = box[0] / 10
    shells = _fcc_shell_vectors(a, 2.5)
    assert len(shells) == 12 + 6 + 24 + 12
    for cells in (False, True):
        o = oracle.forces_cells(x, None, p, pairs=True, lib=lib) if cells else oracle.forces_brute(x, None, p, lib=lib)
        assert o["count"] == 4000 * len(shells) // 2, o["count"]
        assert np.abs(o["F"]).max() < 1e-10
        u_shell = sum(oracle.lj_pair(r, 1.0, 1.0, 2.5, True, lib=lib)[1] for r in shells)
        assert abs(o["U"] / 4000 - 0.5 * u_shell) < 1e-12 * abs(u_shell), (o["U"] / 4000, 0.5 * u_shell)
        w_shell = sum(oracle.lj_pair(r, 1.0, 1.0, 2.5, True, lib=lib)[0] * r * r for r in shells)
        assert abs(o["W"] / 4000 - 0.5 * w_shell) < 1e-11 * abs(w_shell)


def pin_newton3(lib):
    sc = scenarios.fcc_liquid(5, seed=3, jitter=0.15)
    p = _p(sc["box"])
    for cells in (False, True):
        o = oracle.forces_cells(sc["x"], None, p, lib=lib) if cells else oracle.forces_brute(sc["x"], None, p, lib=lib)
        F = o["F"]
        rms = np.sqrt((F * F).sum(1).mean())
        assert np.abs(F.sum(0)).max() <= 1e-12 * len(F) * rms


def pin_virial(lib):
    sc = scenarios.fcc_liquid(4, seed=4, jitter=0.2)
    x, box = sc["x"], sc["box"]
    h = 1e-7
    res = []
    for lam in (1 + h, 1 - h):
        o = oracle.forces_brute(x * lam, None, _p(box * lam, shift=False), lib=lib)
        res.append(o)
    assert res[0]["count"] == res[1]["count"]
    o = oracle.forces_brute(x, None, _p(box, shift=False), lib=lib)
    dudl = (res[0]["U"] - res[1]["U"]) / (2 * h)
    assert abs(o["W"] + dudl) <= 1e-6 * abs(o["W"]), (o["W"], dudl)


def _kdtree_pairs(x, box_len, rc):
    from scipy.spatial import cKDTree
    t = cKDTree(np.mod(x, box_len), boxsize=box_len)
    return oracle.sorted_pairs(np.array(sorted(t.query_pairs(rc)), dtype=np.int64).reshape(-1, 2))


def pin_traversals_agree(lib, seeds=(0, 1, 2)):
    cases = []
    for s in seeds:
        cases.append(scenarios.random_gas(300, 7.0, seed=s, min_dist=0.7))
        cases.append(scenarios.fcc_liquid(3, seed=10 + s, jitter=0.3))
    cases.append(scenarios.random_gas(120, 5.05, seed=7, min_dist=0.7))  # L just above 2 r_c
    for sc in cases:
        x, box = sc["x"], sc["box"]
        p = _p(box)
        b = oracle.forces_brute(x, None, p, pairs=True, lib=lib)
        for cm in (2.5, 1.25, 2.8):
            c = oracle.forces_cells(x, None, p, cell_min=cm, pairs=True, lib=lib)
            assert b["count"] == c["count"], (sc["name"], cm, b["count"], c["count"])
            assert np.array_equal(oracle.sorted_pairs(b["pairs"]), oracle.sorted_pairs(c["pairs"]))
            scale = np.abs(b["F"]).max()
            assert np.abs(b["F"] - c["F"]).max() <= 1e-12 * scale
            assert abs(b["U"] - c["U"]) <= 1e-12 * max(1.0, abs(b["U"]))
        kd = _kdtree_pairs(x, box[0], 2.5)
        mine = oracle.sorted_pairs(b["pairs"])
        if not np.array_equal(kd, mine):
            # tolerate only disagreements within rounding of the cutoff
            a = {tuple(r) for r in kd}
            m = {tuple(r) for r in mine}
            for i, j in a ^ m:
                r2 = oracle.min_image_r2(x[i], x[j], box, lib=lib)
                assert abs(np.sqrt(r2) - 2.5) < 1e-12


def pin_drifted_positions(lib):
    sc = scenarios.fcc_liquid(3, seed=21, jitter=0.3)
    x, box = sc["x"].copy(), sc["box"]
    p = _p(box)
    ref = oracle.forces_brute(x, None, p, pairs=True, lib=lib)
    rng = np.random.default_rng(0)
    # move particles near a face across it by whole box lengths
    y = x.copy()
    for d in range(3):
        lo = y[:, d] < 0.1
        hi = y[:, d] > box[d] - 0.1
        y[lo & (rng.random(len(y)) < 0.5), d] += box[d]
        y[hi & (rng.random(len(y)) < 0.5), d] -= box[d]
    for cm in (2.5, 1.25):
        c = oracle.forces_cells(y, None, p, cell_min=cm, pairs=True, lib=lib)
        b = oracle.forces_brute(y, None, p, pairs=True, lib=lib)
        assert np.array_equal(oracle.sorted_pairs(c["pairs"]), oracle.sorted_pairs(b["pairs"]))
        assert np.array_equal(oracle.sorted_pairs(b["pairs"]), oracle.sorted_pairs(ref["pairs"]))
        assert np.abs(c["F"] - ref["F"]).max() < 1e-9 * np.abs(ref["F"]).max()


def _energy_run(lib, dt, nsteps, ncell=6, seed=1):
    sc = scenarios.fcc_liquid(ncell, seed=seed, jitter=0.05)
    p = _p(sc["box"])
    x, v, ep, ek, _ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], p, dt, nsteps, lib=lib)
    return sc, x, v, ep + ek


def pin_nve(lib):
    sc, x, v, e = _energy_run(lib, 0.005, 100)
    drift = np.abs(e - e[0]).max() / abs(e[0])
    assert drift < 1e-3, drift
    assert np.abs(v.sum(0)).max() < 1e-10
    # Stormer-Verlet energy error is O(dt^2): halving dt quarters it
    _, _, _, e2 = _energy_run(lib, 0.0025, 200)
    d1 = np.abs(e - e[0]).max()
    d2 = np.abs(e2 - e2[0]).max()
    ratio = d1 / d2
    assert 4 * 0.7 < ratio < 4 * 1.3, ratio


def pin_reversibility(lib):
    sc = scenarios.fcc_liquid(4, seed=5, jitter=0.1)
    p = _p(sc["box"])
    x1, v1, *_ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], p, 0.005, 60, lib=lib)
    x2, v2, *_ = oracle.verlet_run(x1, -v1, None, [1.0], p, 0.005, 60, lib=lib)
    L = sc["box"][0]
    d = np.mod(x2 - sc["x"] + 0.5 * L, L) - 0.5 * L
    assert np.abs(d).max() < 1e-9, np.abs(d).max()
    assert np.abs(v2 + sc["v"]).max() < 1e-9


def pin_bin_stats(lib):
    sc = scenarios.fcc_liquid(8, seed=1)
    a = sc["box"][0] / 8
    # bins equal to the conventional cells: 4 sites each (shift off the faces)
    st = oracle.bin_stats(sc["x"] + 0.25 * a, sc["box"], a * 0.999, lib=lib)
    assert st == {"mean": 4.0, "rel_std": 0.0, "median": 4.0, "max": 4.0, "nbins": 512.0, "nempty": 0.0}
    # everything in one bin of 3x3x3 bins
    x = np.full((10, 3), 0.5)
    st = oracle.bin_stats(x, np.full(3, 9.0), 3.0, lib=lib)
    assert st["nbins"] == 27 and st["nempty"] == 26 and st["max"] == 10 and st["median"] == 0
    assert abs(st["mean"] - 10 / 27) < 1e-15
    assert abs(st["rel_std"] - np.std([10] + [0] * 26) / (10 / 27)) < 1e-12
    # even number of bins: median is the mean of the two middle counts
    x = np.array([[0.5, 0.5, 0.5]] * 3 + [[1.5, 0.5, 0.5]])
    st = oracle.bin_stats(x, np.array([2.0, 1.0, 1.0]), 1.0, lib=lib)
    assert st["nbins"] == 2 and st["median"] == 2.0


ALL_PINS = [pin_lj_minimum, pin_lj_shift, pin_lj_scaling_and_gradient, pin_two_body, pin_fcc_lattice,
            pin_newton3, pin_virial, pin_traversals_agree, pin_drifted_positions, pin_nve,
            pin_reversibility, pin_bin_stats]
