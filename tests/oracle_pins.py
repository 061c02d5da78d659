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


# ---------------------------------------------------------------------------
# Gradients (frozen pair mask)


def _mix_params(sc, eps=None, sigma=None, rcut=None, box=None):
    return oracle.make_params(sc["box"] if box is None else box, sc["eps"] if eps is None else eps,
                              sc["sigma"] if sigma is None else sigma, sc["rcut"] if rcut is None else rcut, True)


def pin_vjp_two_body(lib):
    """Closed-form Hessian and parameter derivatives of one isolated pair."""
    rng = np.random.default_rng(11)
    for eps, sig, r in [(1.0, 1.0, 1.05), (1.5, 0.8, 1.3), (0.5, 0.88, 2.0)]:
        d = rng.normal(size=3)
        rhat = d / np.linalg.norm(d)
        x = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0]])
        x[1] -= r * rhat  # x_0 - x_1 = r rhat
        rhat = (x[0] - x[1]) / np.linalg.norm(x[0] - x[1])
        r = np.linalg.norm(x[0] - x[1])
        e = np.array([[0.7, eps], [eps, 1.9]])
        s = np.array([[1.1, sig], [sig, 0.9]])
        p = oracle.make_params(20.0, e, s, 2.5 * s, True)
        types = np.array([0, 1], np.int32)
        # phi(r) = 4 eps (sig^12 r^-12 - sig^6 r^-6) and its r-derivatives
        d1 = 4 * eps * (-12 * sig**12 * r**-13 + 6 * sig**6 * r**-7)
        d2 = 4 * eps * (156 * sig**12 * r**-14 - 42 * sig**6 * r**-8)
        d1_dsig = 4 * eps * (-144 * sig**11 * r**-13 + 36 * sig**5 * r**-7)
        P = np.outer(rhat, rhat)
        H = d2 * P + (d1 / r) * (np.eye(3) - P)
        F0 = -d1 * rhat
        for who in (0, 1):
            c = np.zeros((2, 3))
            c[who] = rng.normal(size=3)
            gx, ge, gs = oracle.force_vjp(x, types, p, [[0, 1]], c, lib=lib)
            # dF_a/dx_b = -d^2U/dx_a dx_b: -H on the diagonal blocks, +H off it
            want = np.zeros((2, 3))
            want[who] = -H @ c[who]
            want[1 - who] = H @ c[who]
            assert np.abs(gx - want).max() < 1e-11 * np.abs(want).max(), (who, gx, want)
            Fw = F0 if who == 0 else -F0
            ge_want = c[who] @ Fw / eps
            gs_want = c[who] @ (-d1_dsig * rhat) * (1 if who == 0 else -1)
            for a, b in ((0, 1), (1, 0)):
                assert abs(ge[a, b] - ge_want) < 1e-12 * abs(ge_want) + 1e-300, (ge, ge_want)
                assert abs(gs[a, b] - gs_want) < 1e-12 * abs(gs_want) + 1e-300, (gs, gs_want)
            assert ge[0, 0] == 0 and ge[1, 1] == 0 and gs[0, 0] == 0 and gs[1, 1] == 0


def pin_vjp_invariants(lib):
    """Translation invariance, Hessian symmetry, eps-linearity, the scaling
    law F(lx; l sigma) = F(x; sigma) / l, and the frozen-list forces equal to
    brute force."""
    sc = scenarios.jittered_mixture(nside=7)
    x, types = sc["x"], sc["types"]
    p = _mix_params(sc)
    ref = oracle.forces_brute(x, types, p, pairs=True, lib=lib)
    pairs = ref["pairs"]
    F = oracle.forces_list(x, types, p, pairs, lib=lib)
    assert np.abs(F - ref["F"]).max() < 1e-12 * np.abs(ref["F"]).max()
    rng = np.random.default_rng(12)
    c = rng.normal(size=x.shape)
    gx, ge, gs = oracle.force_vjp(x, types, p, pairs, c, lib=lib)
    scale = np.abs(gx).sum()
    assert np.abs(gx.sum(0)).max() < 1e-12 * scale, gx.sum(0)
    iu = np.triu_indices(2)
    cF = float((c * F).sum())
    assert abs((sc["eps"][iu] * ge[iu]).sum() - cF) < 1e-11 * abs(cF)
    u = rng.normal(size=x.shape)
    gu = oracle.force_vjp(x, types, p, pairs, u, lib=lib)[0]
    a, b = float((u * gx).sum()), float((c * gu).sum())
    assert abs(a - b) < 1e-11 * (abs(a) + abs(b)), (a, b)
    # Euler identity for the scaling law needs displacements without images:
    # the same cluster placed inside a large box
    xb = x + 10.0
    pb = _mix_params(sc, box=40.0)
    Fb = oracle.forces_list(xb, types, pb, pairs, lib=lib)
    gxb, geb, gsb = oracle.force_vjp(xb, types, pb, pairs, c, lib=lib)
    lhs = (sc["sigma"][iu] * gsb[iu]).sum() + float((xb * gxb).sum())
    rhs = -float((c * Fb).sum())
    assert abs(lhs - rhs) < 1e-10 * abs(rhs), (lhs, rhs)


def _theta_params(sc, eps, sigma, k, h):
    """Parameters with the k-th independent value (eps_00, sig_00, eps_01, ...) scaled by (1 + h)."""
    eps, sigma = eps.copy(), sigma.copy()
    iu = list(zip(*np.triu_indices(eps.shape[0])))
    a, b = iu[k // 2]
    arr = eps if k % 2 == 0 else sigma
    arr[a, b] = arr[b, a] = arr[a, b] * (1.0 + h)
    return _mix_params(sc, eps=eps, sigma=sigma)  # cutoffs unchanged: the mask stays frozen


def _theta_grad(ge, gs):
    return np.array([g[a, b] for a, b in zip(*np.triu_indices(ge.shape[0])) for g in (ge, gs)])


def _theta_vals(sc):
    return _theta_grad(sc["eps"], sc["sigma"])


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def pin_vjp_finite_difference(lib, h=1e-6):
    """Force-matching loss: analytic gradient vs central differences with the
    mask frozen, relative step h for eps/sigma, absolute h for 64 coordinates."""
    sc = scenarios.jittered_mixture(nside=7)
    x, types = sc["x"], sc["types"]
    p = _mix_params(sc)
    et, st, rt = scenarios.perturbed_pair_params(sc["eps"], sc["sigma"])
    Fstar = oracle.forces_cells(x, types, _mix_params(sc, et, st, rt), lib=lib)["F"]
    pairs = oracle.forces_cells(x, types, p, pairs=True, lib=lib)["pairs"]
    L, gx, ge, gs = oracle.force_loss_grad(x, types, p, Fstar, pairs=pairs, lib=lib)
    loss = lambda xx, pp: oracle.force_loss(oracle.forces_list(xx, types, pp, pairs, lib=lib), Fstar)
    th = _theta_vals(sc)
    fd = [(loss(x, _theta_params(sc, sc["eps"], sc["sigma"], k, h)) -
           loss(x, _theta_params(sc, sc["eps"], sc["sigma"], k, -h))) / (2 * h * th[k]) for k in range(6)]
    assert _rel(_theta_grad(ge, gs), fd) < 1e-6, (_theta_grad(ge, gs), fd)
    rng = np.random.default_rng(13)
    idx = [(int(i), int(d)) for i, d in zip(rng.choice(len(x), 64, replace=False), rng.integers(0, 3, 64))]
    fdx, an = [], []
    for i, d in idx:
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        fdx.append((loss(xp, p) - loss(xm, p)) / (2 * h))
        an.append(gx[i, d])
    assert _rel(an, fdx) < 1e-6, _rel(an, fdx)


def _rollout_case(nsteps):
    sc = scenarios.jittered_mixture(nside=7)
    p = _mix_params(sc)
    et, st, rt = scenarios.perturbed_pair_params(sc["eps"], sc["sigma"])
    return sc, p, _mix_params(sc, et, st, rt)


def pin_rollout_finite_difference(lib, nsteps=50, h=1e-6):
    """Gradient of L = mean |F(x_N) - F*_N|^2 through N Verlet steps vs central
    differences of reruns with every time level's mask frozen."""
    sc, p, pt = _rollout_case(nsteps)
    x0, v0, types, mass, dt = sc["x"], sc["v"], sc["types"], sc["mass"], sc["dt"]
    xs_t, *_ = oracle.rollout(x0, v0, types, mass, pt, dt, nsteps, record_masks=False, lib=lib)
    FstarN = oracle.forces_cells(xs_t[nsteps], types, pt, lib=lib)["F"]
    L, gx0, gv0, ge, gs = oracle.rollout_loss_grad(x0, v0, types, mass, p, dt, nsteps, FstarN, lib=lib)
    _, _, masks, off = oracle.rollout(x0, v0, types, mass, p, dt, nsteps, lib=lib)
    mN = masks[off[nsteps]:off[nsteps + 1]]

    def loss(xx, vv, pp):
        xs, *_ = oracle.rollout(xx, vv, types, mass, pp, dt, nsteps, frozen=(masks, off), lib=lib)
        return oracle.force_loss(oracle.forces_list(xs[nsteps], types, pp, mN, lib=lib), FstarN)

    assert abs(loss(x0, v0, p) - L) < 1e-14 * abs(L)
    th = _theta_vals(sc)
    fd = [(loss(x0, v0, _theta_params(sc, sc["eps"], sc["sigma"], k, h)) -
           loss(x0, v0, _theta_params(sc, sc["eps"], sc["sigma"], k, -h))) / (2 * h * th[k]) for k in range(6)]
    assert _rel(_theta_grad(ge, gs), fd) < 1e-6, (_theta_grad(ge, gs), fd)
    rng = np.random.default_rng(14)
    for which, g in (("x", gx0), ("v", gv0)):
        fdx, an = [], []
        for i, d in zip(rng.choice(len(x0), 12, replace=False), rng.integers(0, 3, 12)):
            xp, xm, vp, vm = x0.copy(), x0.copy(), v0.copy(), v0.copy()
            (xp if which == "x" else vp)[i, d] += h
            (xm if which == "x" else vm)[i, d] -= h
            fdx.append((loss(xp, vp, p) - loss(xm, vm, p)) / (2 * h))
            an.append(g[i, d])
        assert _rel(an, fdx) < 1e-6, (which, _rel(an, fdx))


def pin_rollout_symplectic(lib, nsteps=10):
    """The Verlet map is symplectic (unit masses), so is its transpose:
    omega(J^T a, J^T b) = omega(a, b) with omega((x1, v1), (x2, v2)) =
    x1.v2 - v1.x2; zero steps give the identity."""
    sc, p, _ = _rollout_case(nsteps)
    x0, v0, types, dt = sc["x"], sc["v"], sc["types"], sc["dt"]
    rng = np.random.default_rng(15)
    a = rng.normal(size=(2,) + x0.shape)
    b = rng.normal(size=(2,) + x0.shape)
    om = lambda u, w: float((u[0] * w[1]).sum() - (u[1] * w[0]).sum())
    ta = oracle.rollout_vjp(x0, v0, types, [1.0, 1.0], p, dt, nsteps, a[0], a[1], lib=lib)[:2]
    tb = oracle.rollout_vjp(x0, v0, types, [1.0, 1.0], p, dt, nsteps, b[0], b[1], lib=lib)[:2]
    assert abs(om(ta, tb) - om(a, b)) < 1e-10 * np.sqrt(abs(om(ta, ta)) + om(a, b) ** 2 + 1.0), (om(ta, tb), om(a, b))
    assert np.abs(ta[0] - a[0]).max() > 1e-6  # the map is not the identity
    gx, gv, ge, gs = oracle.rollout_vjp(x0, v0, types, [1.0, 1.0], p, dt, 0, a[0], a[1], lib=lib)
    assert np.array_equal(gx, a[0]) and np.array_equal(gv, a[1]) and not ge.any() and not gs.any()


# ---------------------------------------------------------------------------
# Reflective walls and the velocity-scaling thermostat


def pin_walls_free_particle(lib):
    """A lone particle between walls: straight flight, mirrored at each wall
    with the velocity component reversed (closed form: fold x0 + v t)."""
    L, dt, nsteps = 6.0, 0.01, 537
    x0 = np.array([[1.0, 5.5, 3.0]])
    v0 = np.array([[1.3, 0.7, -2.9]])
    p = oracle.make_params(L, 1.0, 1.0, 2.5, True, walls=(1, 1, 1))
    x, v, *_ = oracle.verlet_run(x0, v0, None, [1.0], p, dt, nsteps, lib=lib)
    u = x0 + v0 * dt * nsteps
    k = np.floor(u / L)
    folded = np.where(k % 2 == 0, u - k * L, (k + 1) * L - u)
    assert np.abs(x - folded).max() < 1e-9, (x, folded)
    assert np.allclose(v, np.where(k % 2 == 0, v0, -v0))


def pin_walls_pairs_and_forces(lib):
    """Between walls no pair is taken through a face: the brute-force pair set
    equals scipy's non-periodic k-d tree, and brute force equals linked cells.
    With walls in x only, y and z keep their minimum images."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(21)
    L = 9.0
    x = rng.uniform(0.0, L, (300, 3))
    p = oracle.make_params(L, 1.0, 1.0, 2.5, True, walls=(1, 1, 1))
    b = oracle.forces_brute(x, None, p, pairs=True, lib=lib)
    ref = cKDTree(x).query_pairs(2.5, output_type="ndarray")
    assert np.array_equal(oracle.sorted_pairs(b["pairs"]), oracle.sorted_pairs(ref))
    c = oracle.forces_cells(x, None, p, pairs=True, lib=lib)
    assert np.array_equal(oracle.sorted_pairs(c["pairs"]), oracle.sorted_pairs(ref))
    assert np.abs(b["F"] - c["F"]).max() < 1e-9 * np.abs(b["F"]).max()
    # mixed: walls in x, periodic y and z: distances use images in y, z only
    p2 = oracle.make_params(L, 1.0, 1.0, 2.5, True, walls=(1, 0, 0))
    b2 = oracle.forces_brute(x, None, p2, pairs=True, lib=lib)
    d = x[:, None, :] - x[None, :, :]
    d[..., 1:] -= L * np.round(d[..., 1:] / L)
    r2 = (d * d).sum(-1)
    iu = np.triu_indices(len(x), 1)
    want = np.stack(iu, 1)[r2[iu] < 6.25]
    assert np.array_equal(oracle.sorted_pairs(b2["pairs"]), oracle.sorted_pairs(want))
    c2 = oracle.forces_cells(x, None, p2, pairs=True, lib=lib)
    assert np.array_equal(oracle.sorted_pairs(c2["pairs"]), oracle.sorted_pairs(want))


def pin_walls_nve(lib):
    """Elastic walls conserve the energy of a liquid in a closed box."""
    x, box = scenarios.fcc_lattice(4, 0.7)
    L = box[0] + 1.0  # a gap at the walls
    x = x + 0.5
    rng = np.random.default_rng(22)
    v = scenarios.maxwell_boltzmann(len(x), 1.5, 1.0, rng)
    p = oracle.make_params(L, 1.0, 1.0, 2.5, True, walls=(1, 1, 1))
    _, _, ep, ek, _ = oracle.verlet_run(x, v, None, [1.0], p, 0.002, 300, lib=lib)
    e = ep + ek
    assert np.abs(e - e[0]).max() < 2e-3 * abs(ek[0]), np.abs(e - e[0]).max()


def pin_thermostat(lib):
    """One scaling step reaches the target within the allowed change, or
    moves exactly by the allowed change; dof 3N between walls, 3N - 3 in a
    periodic box."""
    rng = np.random.default_rng(23)
    v = rng.normal(0.0, 1.0, (500, 3))
    for walls, dof in (((0, 0, 0), 1497), ((1, 1, 1), 1500)):
        p = oracle.make_params(10.0, 1.0, 1.0, 2.5, True, walls=walls)
        t0 = (v * v).sum() / dof
        v1, tb = oracle.thermostat(v, None, [1.0], p, t0 + 0.05, 0.1, lib=lib)
        assert abs(tb - t0) < 1e-12 * t0 and abs((v1 * v1).sum() / dof - (t0 + 0.05)) < 1e-12
        v2, _ = oracle.thermostat(v, None, [1.0], p, t0 + 5.0, 0.1, lib=lib)
        assert abs((v2 * v2).sum() / dof - (t0 + 0.1)) < 1e-12
        assert np.allclose(v2 / v, v2[0, 0] / v[0, 0])  # one common factor


ALL_PINS = [pin_lj_minimum, pin_lj_shift, pin_lj_scaling_and_gradient, pin_two_body, pin_fcc_lattice,
            pin_newton3, pin_virial, pin_traversals_agree, pin_drifted_positions, pin_nve,
            pin_reversibility, pin_bin_stats, pin_vjp_two_body, pin_vjp_invariants,
            pin_vjp_finite_difference, pin_rollout_finite_difference, pin_rollout_symplectic,
            pin_walls_free_particle, pin_walls_pairs_and_forces, pin_walls_nve, pin_thermostat]
