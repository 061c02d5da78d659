"""torch.autograd bindings of the force VJP and the checkpointed rollout adjoint.

Marshalling only: every derivative is computed by the library's kernels
(``ljsel_force_vjp``, ``ljsel_rollout_vjp``).  Positions and velocities are
(n, 3) float64 CUDA tensors in the caller's order; eps and sigma are
(ntypes, ntypes) float64 tensors (symmetric); with ``rcut_factor`` the
cutoffs follow as rcut_factor * sigma, otherwise the system's cutoffs stay.
The pair set is frozen at each evaluation point (derivatives almost
everywhere), as the library defines.  The library returns, for a != b, the
derivative with respect to the shared parameter eps_ab = eps_ba; the
gradient of the (ntypes, ntypes) tensor puts half of it on each of the two
entries, so that a symmetric tensor built from independent values receives
the full derivative through the chain rule.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ljsel_compute, ljsel_force_vjp, ljsel_get_state, ljsel_rollout_vjp, ljsel_set_state

__all__ = ["LJForces", "LJRollout", "forces", "rollout"]


def _split(g, like):
    g = np.array(g, np.float64)
    off = ~np.eye(g.shape[0], dtype=bool)
    g[off] *= 0.5
    return torch.from_numpy(g).to(like)


def _load(system, pos, eps, sigma, rcut_factor, vel=None):
    e = eps.detach().double().cpu().numpy()
    s = sigma.detach().double().cpu().numpy()
    system.set_pair_params(e, s, None if rcut_factor is None else rcut_factor * s)
    ljsel_set_state(system.h, pos.detach().contiguous(), None if vel is None else vel.detach().contiguous())


class LJForces(torch.autograd.Function):
    """F(x; eps, sigma) with gradients w.r.t. x (Hessian-vector products) and eps/sigma."""

    @staticmethod
    def forward(ctx, system, pos, eps, sigma, rcut_factor=None):
        _load(system, pos, eps, sigma, rcut_factor)
        F = torch.empty_like(pos)
        ljsel_compute(system.h, F)
        ctx.system, ctx.rcut_factor = system, rcut_factor
        ctx.save_for_backward(pos, eps, sigma)
        return F

    @staticmethod
    def backward(ctx, gF):
        pos, eps, sigma = ctx.saved_tensors
        system = ctx.system
        _load(system, pos, eps, sigma, ctx.rcut_factor)
        gpos = torch.empty_like(pos)
        ge, gs = ljsel_force_vjp(system.h, gF.contiguous(), gpos, system.ntypes)
        return None, gpos, _split(ge, eps), _split(gs, sigma), None


class LJRollout(torch.autograd.Function):
    """(x_N, v_N) after N Stormer-Verlet steps from (x_0, v_0), differentiable
    w.r.t. x_0, v_0, eps and sigma through checkpoints every ``every`` steps."""

    @staticmethod
    def forward(ctx, system, x0, v0, eps, sigma, nsteps, every, rcut_factor=None):
        _load(system, x0, eps, sigma, rcut_factor, v0)
        system.rollout(nsteps, every)
        xN, vN = torch.empty_like(x0), torch.empty_like(v0)
        ljsel_get_state(system.h, xN, vN)
        token = object()
        system._rollout_token = token
        ctx.system, ctx.token, ctx.args = system, token, (nsteps, every, rcut_factor)
        ctx.save_for_backward(x0, v0, eps, sigma)
        return xN, vN

    @staticmethod
    def backward(ctx, gx, gv):
        x0, v0, eps, sigma = ctx.saved_tensors
        system = ctx.system
        nsteps, every, rcut_factor = ctx.args
        e = eps.detach().double().cpu().numpy()
        s = sigma.detach().double().cpu().numpy()
        system.set_pair_params(e, s, None if rcut_factor is None else rcut_factor * s)
        if getattr(system, "_rollout_token", None) is not ctx.token or not system.has_rollout():
            # another rollout, or a parameter change, replaced this one: record it again
            _load(system, x0, eps, sigma, rcut_factor, v0)
            system.rollout(nsteps, every)
            system._rollout_token = ctx.token
        gx = torch.zeros_like(x0) if gx is None else gx.contiguous()
        gv = None if gv is None else gv.contiguous()
        gx0, gv0 = torch.empty_like(x0), torch.empty_like(v0)
        ge, gs = ljsel_rollout_vjp(system.h, gx, gv, gx0, gv0, system.ntypes)
        return None, gx0, gv0, _split(ge, eps), _split(gs, sigma), None, None, None


def forces(system, pos, eps, sigma, rcut_factor=None):
    return LJForces.apply(system, pos, eps, sigma, rcut_factor)


def rollout(system, x0, v0, eps, sigma, nsteps, every, rcut_factor=None):
    return LJRollout.apply(system, x0, v0, eps, sigma, nsteps, every, rcut_factor)
