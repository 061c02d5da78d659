"""GPU gradients (force VJP, checkpointed rollout adjoint) against the FP64 oracle.

The differentiable binary mixture (80:20, eps/sigma of the Kob-Andersen
type, r_c,ab = 2.5 sigma_ab, density 1.2): a jittered 7^3 lattice (N = 343)
for the element-wise and finite-difference checks, the full 32^3 lattice
(N = 32,768) for parity at size.  The pair mask is frozen at every
evaluation point on both sides.  FP64 path: equal to the oracle's analytic
gradient within 1e-10 (one step) / 1e-9 (50 steps) relative, and to central
differences (h = 1e-6) within 1e-6.  FP32 path: the 50-step rollout
gradient within 5e-4 relative of the FP64 oracle (measured about 5e-5: FP32
rounding of the forces, 1e-6 relative, grows through the chaotic dynamics
over 0.25 time units; the bar leaves a factor 10).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2505_03438_gb300 as lj
from paper_2505_03438_gb300 import scenarios

pytestmark = pytest.mark.gpu


def _op(sc, eps=None, sigma=None, rcut=None):
    return oracle.make_params(sc["box"], sc["eps"] if eps is None else eps, sc["sigma"] if sigma is None else sigma,
                              sc["rcut"] if rcut is None else rcut, True)


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _theta(ge, gs):
    return np.array([g[a, b] for a, b in zip(*np.triu_indices(ge.shape[0])) for g in (ge, gs)])


def _theta_torch(eg, sg):
    """Shared-parameter derivatives from torch gradients of symmetric (nt, nt) tensors."""
    return _theta(eg + eg.T - np.diag(np.diag(eg)), sg + sg.T - np.diag(np.diag(sg)))


def _case(size):
    return scenarios.jittered_mixture(nside=7) if size == "small" else scenarios.binary_mixture()


@pytest.mark.parametrize("precision", [1, 0], ids=["fp64", "fp32"])
@pytest.mark.parametrize("size,cfg", [("small", None), ("full", None), ("small", dict(method="LC")),
                                      ("full", dict(method="LC")), ("small", dict(method="VL", newton3=True)),
                                      ("small", dict(method="VL", csf=0.5)), ("small", dict(method="LC", csf=0.5))],
                         ids=["small-rows", "full-rows", "small-cells", "full-cells", "small-n3l-cells",
                              "small-rows-csf0.5", "small-cells-csf0.5"])
def test_force_vjp_matches_oracle(size, cfg, precision):
    """Verlet-list rows (VL without N3L) and the cell traversal (every other
    configuration) give the same VJP as the oracle."""
    sc = _case(size)
    x, types = sc["x"], sc["types"]
    s = lj.System(sc, precision=precision)
    if cfg:
        s.set_config(rebuild_interval=10, **cfg)
    c = np.random.default_rng(21).normal(size=x.shape)
    g, ge, gs = s.force_vjp(c)
    xo = x if precision else _f32(x)  # the positions the GPU pair arithmetic works on
    p = _op(sc)
    pairs = oracle.forces_cells(xo, types, p, pairs=True)["pairs"]
    go, geo, gso = oracle.force_vjp(xo, types, p, pairs, c)
    tol = 1e-10 if precision else 1e-5
    assert _rel(g, go) < tol, ("positions", _rel(g, go))
    assert _rel(_theta(ge, gs), _theta(geo, gso)) < tol, (_theta(ge, gs), _theta(geo, gso))
    # symmetric entries hold the same shared-parameter derivative
    assert abs(ge[0, 1] - ge[1, 0]) <= 1e-12 * abs(ge[0, 1]) and abs(gs[0, 1] - gs[1, 0]) <= 1e-12 * abs(gs[0, 1])


def test_force_vjp_finite_differences_fp64(h=1e-6):
    """dL/d(eps, sigma) and dL/dx of the force-matching loss vs central
    differences of the GPU's own FP64 loss, cutoffs held fixed so that the
    pair set stays frozen."""
    sc = _case("small")
    x, v, types = sc["x"], sc["v"], sc["types"]
    s = lj.System(sc, precision=1)
    et, st, rt = scenarios.perturbed_pair_params(sc["eps"], sc["sigma"])
    Fstar = oracle.forces_cells(x, types, _op(sc, et, st, rt))["F"]
    F0 = s.compute()[0]
    g, ge, gs = s.force_vjp(2.0 * (F0 - Fstar) / F0.size)
    loss = lambda: oracle.force_loss(s.compute()[0], Fstar)
    npairs = s.pairs()[1]
    fd = []
    iu = list(zip(*np.triu_indices(2)))
    for k in range(6):
        a, b = iu[k // 2]
        vals = []
        for sgn in (1, -1):
            e, sg = sc["eps"].copy(), sc["sigma"].copy()
            arr = e if k % 2 == 0 else sg
            th = arr[a, b]
            arr[a, b] = arr[b, a] = th * (1 + sgn * h)
            s.set_pair_params(e, sg, sc["rcut"])
            vals.append(loss())
        fd.append((vals[0] - vals[1]) / (2 * h * th))
    s.set_pair_params(sc["eps"], sc["sigma"], sc["rcut"])
    assert _rel(_theta(ge, gs), fd) < 1e-6, (_theta(ge, gs), fd)
    rng = np.random.default_rng(22)
    an, fdx = [], []
    for i, d in zip(rng.choice(len(x), 16, replace=False), rng.integers(0, 3, 16)):
        vals = []
        for sgn in (1, -1):
            xx = x.copy()
            xx[i, d] += sgn * h
            s.set_state(xx, v)
            assert s.pairs()[1] == npairs
            vals.append(loss())
        fdx.append((vals[0] - vals[1]) / (2 * h))
        an.append(g[i, d])
    assert _rel(an, fdx) < 1e-6, _rel(an, fdx)


def _torch(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_autograd_force_loss_fp64():
    sc = _case("small")
    x, types = sc["x"], sc["types"]
    et, st, rt = scenarios.perturbed_pair_params(sc["eps"], sc["sigma"])
    Fstar = oracle.forces_cells(x, types, _op(sc, et, st, rt))["F"]
    s = lj.System(sc, precision=1)
    from paper_2505_03438_gb300 import autograd as A
    xt = _torch(x).requires_grad_(True)
    eps = torch.tensor(sc["eps"], dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(sc["sigma"], dtype=torch.float64, requires_grad=True)
    F = A.forces(s, xt, eps, sig, 2.5)
    L = ((F - _torch(Fstar)) ** 2).mean()
    L.backward()
    Lo, gxo, geo, gso = oracle.force_loss_grad(x, types, _op(sc), Fstar)
    assert abs(L.item() - Lo) < 1e-12 * Lo
    assert _rel(xt.grad.cpu().numpy(), gxo) < 1e-10
    # torch sees eps_ab and eps_ba as two entries: their grads add up to the shared derivative
    assert _rel(_theta_torch(eps.grad.numpy(), sig.grad.numpy()), _theta(geo, gso)) < 1e-10


def _rollout_grads(s, sc, nsteps, every, Fstar_end):
    from paper_2505_03438_gb300 import autograd as A
    x0 = _torch(sc["x"]).requires_grad_(True)
    v0 = _torch(sc["v"]).requires_grad_(True)
    eps = torch.tensor(sc["eps"], dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(sc["sigma"], dtype=torch.float64, requires_grad=True)
    xN, vN = A.rollout(s, x0, v0, eps, sig, nsteps, every, 2.5)
    F = A.forces(s, xN, eps, sig, 2.5)
    L = ((F - _torch(Fstar_end)) ** 2).mean()
    L.backward()
    return (L.item(), x0.grad.cpu().numpy(), v0.grad.cpu().numpy(),
            _theta_torch(eps.grad.numpy(), sig.grad.numpy()))


def _oracle_rollout(sc, nsteps):
    types, mass, dt = sc["types"], sc["mass"], sc["dt"]
    et, st, rt = scenarios.perturbed_pair_params(sc["eps"], sc["sigma"])
    pt = _op(sc, et, st, rt)
    xs_t, *_ = oracle.rollout(sc["x"], sc["v"], types, mass, pt, dt, nsteps, record_masks=False)
    FstarN = oracle.forces_cells(xs_t[nsteps], types, pt)["F"]
    L, gx, gv, ge, gs = oracle.rollout_loss_grad(sc["x"], sc["v"], types, mass, _op(sc), dt, nsteps, FstarN)
    return FstarN, (L, gx, gv, _theta(ge, gs))


@pytest.fixture(scope="module")
def small_rollout_oracle():
    sc = _case("small")
    return sc, _oracle_rollout(sc, 50)


@pytest.mark.parametrize("precision", [1, 0], ids=["fp64", "fp32"])
def test_rollout_gradient_matches_oracle(small_rollout_oracle, precision):
    sc, (FstarN, ref) = small_rollout_oracle
    s = lj.System(sc, precision=precision)
    got = _rollout_grads(s, sc, 50, 10, FstarN)
    tol = 1e-9 if precision else 5e-4
    assert abs(got[0] - ref[0]) < tol * ref[0], (got[0], ref[0])
    for name, a, b in zip(("x0", "v0", "theta"), got[1:], ref[1:]):
        assert _rel(a, b) < tol, (name, _rel(a, b))


def test_rollout_checkpoint_spacing_fp64(small_rollout_oracle):
    """The gradient does not depend on where the checkpoints sit."""
    sc, (FstarN, ref) = small_rollout_oracle
    s = lj.System(sc, precision=1)
    base = _rollout_grads(s, sc, 50, 10, FstarN)
    for every in (1, 7, 50, 64):
        got = _rollout_grads(s, sc, 50, every, FstarN)
        for a, b in zip(got[1:], base[1:]):
            assert _rel(a, b) < 1e-12, every


def test_rollout_vjp_edges():
    sc = _case("small")
    s = lj.System(sc, precision=1)
    with pytest.raises(lj.LjselError):
        s.rollout_vjp(np.zeros((s.n, 3)))
    s.rollout(0, 10)
    a = np.random.default_rng(23).normal(size=(2, s.n, 3))
    gx, gv, ge, gs = s.rollout_vjp(a[0], a[1])
    assert np.array_equal(gx, a[0]) and np.array_equal(gv, a[1]) and not ge.any() and not gs.any()
    # after the reverse pass the system sits at the rollout's final state
    s.rollout(20, 8)
    xe, ve = s.state()
    s.rollout_vjp(a[0], a[1])
    xa, va = s.state()
    assert np.array_equal(xe, xa) and np.array_equal(ve, va)
    # a parameter change drops the record
    s.set_pair_params(sc["eps"] * 1.01, sc["sigma"])
    with pytest.raises(lj.LjselError):
        s.rollout_vjp(a[0], a[1])


@pytest.mark.slow
def test_rollout_gradient_full_size():
    """N = 32,768, 50 steps, checkpoints every 10: FP64 path against the
    oracle's analytic gradient, FP32 path error bounded."""
    sc = _case("full")
    FstarN, ref = _oracle_rollout(sc, 50)
    for precision, tol in ((1, 1e-9), (0, 5e-4)):
        s = lj.System(sc, precision=precision)
        got = _rollout_grads(s, sc, 50, 10, FstarN)
        assert abs(got[0] - ref[0]) < tol * ref[0], (precision, got[0], ref[0])
        for name, a, b in zip(("x0", "v0", "theta"), got[1:], ref[1:]):
            assert _rel(a, b) < tol, (precision, name, _rel(a, b))
        s.close()
