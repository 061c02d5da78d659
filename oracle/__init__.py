"""FP64 CPU oracle for the cutoff Lennard-Jones hot path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference arm of ``bench.py`` may import this package.  The GPU library never
imports it, and this package imports nothing from the GPU library: the two
share only the seeded input generators, which hold none of the method's
arithmetic.

The arithmetic lives in ``ljoracle.c`` (plain C, FP64, ``-ffp-contract=off``);
this module only compiles it with gcc and marshals numpy arrays through
ctypes.  Each wrapper names the paper section its C routine follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ljoracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libljoracle.so")
_LOCK = threading.Lock()
_LIB = None

MAX_TYPES = 4


def build(force: bool = False, src: str = _SRC, out: str = _SO, extra=()) -> str:
    """Compile the oracle with gcc (OpenMP, no fused multiply-add)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", *extra, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class Params(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("ntypes", ctypes.c_int32),
        ("shift", ctypes.c_int32),
        ("eps", ctypes.c_double * (MAX_TYPES * MAX_TYPES)),
        ("sigma", ctypes.c_double * (MAX_TYPES * MAX_TYPES)),
        ("rcut", ctypes.c_double * (MAX_TYPES * MAX_TYPES)),
        ("walls", ctypes.c_int32 * 3),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)


def _bind(lib):
    lib.orc_lj_pair.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int32, _D, _D]
    lib.orc_lj_pair.restype = None
    lib.orc_min_image_r2.argtypes = [ctypes.c_double] * 6 + [_D, _D]
    lib.orc_min_image_r2.restype = None
    lib.orc_forces_brute.argtypes = [ctypes.c_int64, _D, _I32, ctypes.POINTER(Params), _D, _D, _D, _I32, ctypes.c_int64]
    lib.orc_forces_brute.restype = ctypes.c_int64
    lib.orc_forces_cells.argtypes = [ctypes.c_int64, _D, _I32, ctypes.POINTER(Params), ctypes.c_double, ctypes.c_int32,
                                     _D, _D, _D, _I32, ctypes.c_int64]
    lib.orc_forces_cells.restype = ctypes.c_int64
    lib.orc_verlet_run.argtypes = [ctypes.c_int64, _D, _D, _I32, _D, ctypes.POINTER(Params), ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int64, ctypes.c_int32, _D, _D, _D]
    lib.orc_verlet_run.restype = ctypes.c_int32
    lib.orc_bin_stats.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, _D]
    lib.orc_bin_stats.restype = None
    lib.orc_forces_list.argtypes = [ctypes.c_int64, _D, _I32, ctypes.POINTER(Params), _I32, ctypes.c_int64, _D]
    lib.orc_forces_list.restype = None
    lib.orc_force_vjp.argtypes = [ctypes.c_int64, _D, _I32, ctypes.POINTER(Params), _I32, ctypes.c_int64, _D,
                                  _D, _D, _D]
    lib.orc_force_vjp.restype = None
    lib.orc_rollout.argtypes = [ctypes.c_int64, _D, _D, _I32, _D, ctypes.POINTER(Params), ctypes.c_double,
                                ctypes.c_int64, _D, _D, _I32, _I64, _I32, ctypes.c_int64, _I64]
    lib.orc_rollout.restype = ctypes.c_int64
    lib.orc_rollout_vjp.argtypes = [ctypes.c_int64, _D, _D, _I32, _D, ctypes.POINTER(Params), ctypes.c_double,
                                    ctypes.c_int64, _D, _D, _D, _D, _D, _D]
    lib.orc_rollout_vjp.restype = None
    lib.orc_thermostat.argtypes = [ctypes.c_int64, _D, _I32, _D, ctypes.POINTER(Params), ctypes.c_double,
                                   ctypes.c_double]
    lib.orc_thermostat.restype = ctypes.c_double
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle library; a custom path loads a variant."""
    global _LIB
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _LOCK:
        if _LIB is None:
            _LIB = _bind(ctypes.CDLL(build()))
    return _LIB


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I32)


def make_params(box, eps, sigma, rcut, shift=True, walls=(0, 0, 0)) -> Params:
    """Pack a parameter set.  eps/sigma/rcut: scalars (one type) or ntypes x ntypes;
    walls[d] = 1 closes dimension d with reflective walls (no periodic image)."""
    eps = np.atleast_2d(np.asarray(eps, dtype=np.float64))
    sigma = np.atleast_2d(np.asarray(sigma, dtype=np.float64))
    nt = eps.shape[0]
    rcut = np.asarray(rcut, dtype=np.float64)
    if rcut.ndim == 0:
        rcut = np.full((nt, nt), float(rcut))
    p = Params()
    box = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    for d in range(3):
        p.box[d] = float(box[d])
    p.ntypes = nt
    p.shift = 1 if shift else 0
    for d in range(3):
        p.walls[d] = 1 if walls[d] else 0
    for a in range(nt):
        for b in range(nt):
            p.eps[a * nt + b] = float(eps[a, b])
            p.sigma[a * nt + b] = float(sigma[a, b])
            p.rcut[a * nt + b] = float(rcut[a, b])
    return p


def lj_pair(r, eps=1.0, sigma=1.0, rc=2.5, shift=True, lib=None):
    """(f_over_r, u) of one pair at distance r (Sec. 2.1)."""
    lib = lib or load()
    f = ctypes.c_double()
    u = ctypes.c_double()
    lib.orc_lj_pair(float(r), float(eps), float(sigma), float(rc), 1 if shift else 0, ctypes.byref(f), ctypes.byref(u))
    return f.value, u.value


def min_image_r2(xi, xj, box, lib=None):
    lib = lib or load()
    out = ctypes.c_double()
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, np.float64), (3,)))
    lib.orc_min_image_r2(*[float(v) for v in xi], *[float(v) for v in xj], _dp(b), ctypes.byref(out))
    return out.value


def _prep(x, types):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    if types is None:
        types = np.zeros(n, np.int32)
    types = np.ascontiguousarray(types, dtype=np.int32)
    return x, types, n


def forces_brute(x, types, params: Params, pairs=False, lib=None):
    """O(N^2) minimum-image forces, energy, virial and pair set (Sec. 2.1)."""
    lib = lib or load()
    x, types, n = _prep(x, types)
    F = np.zeros((n, 3))
    U = ctypes.c_double()
    W = ctypes.c_double()
    cap = 0
    buf = None
    if pairs:
        cap = lib.orc_forces_brute(n, _dp(x), _ip(types), ctypes.byref(params), _dp(F), None, None, None, 0)
        buf = np.zeros((max(cap, 1), 2), np.int32)
    cnt = lib.orc_forces_brute(n, _dp(x), _ip(types), ctypes.byref(params), _dp(F), ctypes.byref(U), ctypes.byref(W),
                               _ip(buf) if pairs else None, cap)
    out = {"F": F, "U": U.value, "W": W.value, "count": int(cnt)}
    if pairs:
        out["pairs"] = buf[:cnt]
    return out


def forces_cells(x, types, params: Params, cell_min=None, nthreads=0, pairs=False, lib=None):
    """Linked-cell forces, energy, virial and pair set (Sec. 2.2.1)."""
    lib = lib or load()
    x, types, n = _prep(x, types)
    if cell_min is None:
        nt = params.ntypes
        cell_min = max(params.rcut[k] for k in range(nt * nt))
    F = np.zeros((n, 3))
    U = ctypes.c_double()
    W = ctypes.c_double()
    cap = 0
    buf = None
    if pairs:
        cap = lib.orc_forces_cells(n, _dp(x), _ip(types), ctypes.byref(params), float(cell_min), int(nthreads),
                                   _dp(F), None, None, None, 0)
        buf = np.zeros((max(cap, 1), 2), np.int32)
    cnt = lib.orc_forces_cells(n, _dp(x), _ip(types), ctypes.byref(params), float(cell_min), int(nthreads),
                               _dp(F), ctypes.byref(U), ctypes.byref(W), _ip(buf) if pairs else None, cap)
    out = {"F": F, "U": U.value, "W": W.value, "count": int(cnt)}
    if pairs:
        out["pairs"] = buf[:cnt]
    return out


def verlet_run(x, v, types, mass, params: Params, dt, nsteps, cell_min=None, nthreads=0, lib=None):
    """Velocity-form Stormer-Verlet trajectory (Sec. 2.1).  Returns (x, v, epot, ekin, vir)."""
    lib = lib or load()
    x, types, n = _prep(x, types)
    x = x.copy()
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3).copy()
    mass = np.ascontiguousarray(np.atleast_1d(np.asarray(mass, np.float64)))
    if cell_min is None:
        nt = params.ntypes
        cell_min = max(params.rcut[k] for k in range(nt * nt))
    ep = np.zeros(nsteps + 1)
    ek = np.zeros(nsteps + 1)
    vr = np.zeros(nsteps + 1)
    rc = lib.orc_verlet_run(n, _dp(x), _dp(v), _ip(types), _dp(mass), ctypes.byref(params), float(cell_min),
                            float(dt), int(nsteps), int(nthreads), _dp(ep), _dp(ek), _dp(vr))
    if rc != 0:
        raise MemoryError("oracle verlet_run failed")
    return x, v, ep, ek, vr


def bin_stats(x, box, bin_min, lib=None):
    """Live statistics over CSF-1 cell bins (Sec. 4): dict of the six counts statistics."""
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, np.float64), (3,)))
    out = np.zeros(6)
    lib.orc_bin_stats(x.shape[0], _dp(x), _dp(b), float(bin_min), _dp(out))
    return dict(zip(["mean", "rel_std", "median", "max", "nbins", "nempty"], out.tolist()))


def sorted_pairs(p):
    """Canonical (lexicographically sorted, i < j) pair array for set comparison."""
    p = np.asarray(p, dtype=np.int64).reshape(-1, 2)
    lo = np.minimum(p[:, 0], p[:, 1])
    hi = np.maximum(p[:, 0], p[:, 1])
    order = np.lexsort((hi, lo))
    return np.stack([lo[order], hi[order]], 1)


# ---------------------------------------------------------------------------
# Gradients (the differentiable binary-mixture workload; the pair mask is
# frozen at the evaluation point, see ljoracle.c)


def _pairs_arr(pairs):
    return np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))


def forces_list(x, types, params: Params, pairs, lib=None):
    """Forces over a fixed list of unordered pairs (frozen mask), minimum image."""
    lib = lib or load()
    x, types, n = _prep(x, types)
    pr = _pairs_arr(pairs)
    F = np.zeros((n, 3))
    lib.orc_forces_list(n, _dp(x), _ip(types), ctypes.byref(params), _ip(pr), pr.shape[0], _dp(F))
    return F


def force_vjp(x, types, params: Params, pairs, cot, lib=None):
    """(dF/dx)^T cot and d(cot . F)/d(eps, sigma) over a frozen pair list.

    Returns (gx [n, 3], geps [nt, nt], gsig [nt, nt]); entries (a, b) and
    (b, a) of geps/gsig both hold the derivative for the shared parameter.
    """
    lib = lib or load()
    x, types, n = _prep(x, types)
    pr = _pairs_arr(pairs)
    c = np.ascontiguousarray(cot, dtype=np.float64).reshape(n, 3)
    nt = params.ntypes
    gx = np.zeros((n, 3))
    ge = np.zeros(nt * nt)
    gs = np.zeros(nt * nt)
    lib.orc_force_vjp(n, _dp(x), _ip(types), ctypes.byref(params), _ip(pr), pr.shape[0], _dp(c),
                      _dp(gx), _dp(ge), _dp(gs))
    return gx, ge.reshape(nt, nt), gs.reshape(nt, nt)


def rollout(x0, v0, types, mass, params: Params, dt, nsteps, frozen=None, record_masks=True, lib=None):
    """Unwrapped velocity-form Stormer-Verlet (Sec. 2.1) for gradient checks.

    Returns (xs [nsteps+1, n, 3], vs [...], masks, offsets): with ``frozen``
    = (masks, offsets) of an earlier run the pair mask of every time level is
    taken from it instead of being recomputed; without ``record_masks`` the
    masks are not kept (masks, offsets are None).
    """
    lib = lib or load()
    x0, types, n = _prep(x0, types)
    v0 = np.ascontiguousarray(v0, dtype=np.float64).reshape(n, 3)
    mass = np.ascontiguousarray(np.atleast_1d(np.asarray(mass, np.float64)))
    xs = np.zeros((nsteps + 1, n, 3))
    vs = np.zeros((nsteps + 1, n, 3))
    if frozen is not None:
        masks, off = _pairs_arr(frozen[0]), np.ascontiguousarray(frozen[1], dtype=np.int64)
        lib.orc_rollout(n, _dp(x0), _dp(v0), _ip(types), _dp(mass), ctypes.byref(params), float(dt), int(nsteps),
                        _dp(xs), _dp(vs), _ip(masks), off.ctypes.data_as(_I64), None, 0, None)
        return xs, vs, masks, off
    if not record_masks:
        lib.orc_rollout(n, _dp(x0), _dp(v0), _ip(types), _dp(mass), ctypes.byref(params), float(dt), int(nsteps),
                        _dp(xs), _dp(vs), None, None, None, 0, None)
        return xs, vs, None, None
    off = np.zeros(nsteps + 2, np.int64)
    cap = int(forces_cells(x0, types, params, lib=lib)["count"] * 1.25 * (nsteps + 1)) + 1024
    masks = np.zeros((cap, 2), np.int32)
    for _ in range(2):
        total = lib.orc_rollout(n, _dp(x0), _dp(v0), _ip(types), _dp(mass), ctypes.byref(params), float(dt),
                                int(nsteps), _dp(xs), _dp(vs), None, None, _ip(masks), cap,
                                off.ctypes.data_as(_I64))
        if total <= cap:
            return xs, vs, masks[:total], off
        cap = int(total)
        masks = np.zeros((cap, 2), np.int32)
    raise RuntimeError("rollout masks changed between two identical runs")


def rollout_vjp(x0, v0, types, mass, params: Params, dt, nsteps, xbar, vbar, lib=None):
    """Cotangents of (x_0, v_0, eps, sigma) from those of (x_N, v_N) through N steps."""
    lib = lib or load()
    x0, types, n = _prep(x0, types)
    v0 = np.ascontiguousarray(v0, dtype=np.float64).reshape(n, 3)
    mass = np.ascontiguousarray(np.atleast_1d(np.asarray(mass, np.float64)))
    xb = np.ascontiguousarray(xbar, dtype=np.float64).reshape(n, 3)
    vb = np.ascontiguousarray(vbar, dtype=np.float64).reshape(n, 3)
    nt = params.ntypes
    gx, gv = np.zeros((n, 3)), np.zeros((n, 3))
    ge, gs = np.zeros(nt * nt), np.zeros(nt * nt)
    lib.orc_rollout_vjp(n, _dp(x0), _dp(v0), _ip(types), _dp(mass), ctypes.byref(params), float(dt), int(nsteps),
                        _dp(xb), _dp(vb), _dp(gx), _dp(gv), _dp(ge), _dp(gs))
    return gx, gv, ge.reshape(nt, nt), gs.reshape(nt, nt)


def force_loss(F, Fstar):
    """Mean squared force difference L = sum |F - F*|^2 / (3N)."""
    d = np.asarray(F) - np.asarray(Fstar)
    return float((d * d).sum() / d.size)


def force_loss_grad(x, types, params: Params, Fstar, pairs=None, lib=None):
    """Loss and its gradient w.r.t. positions and (eps, sigma) at one configuration.

    The pair mask is that of x under ``params`` unless ``pairs`` is given.
    Returns (L, gx, geps, gsig).
    """
    lib = lib or load()
    if pairs is None:
        pairs = forces_cells(x, types, params, pairs=True, lib=lib)["pairs"]
    F = forces_list(x, types, params, pairs, lib=lib)
    cot = 2.0 * (F - Fstar) / F.size
    gx, ge, gs = force_vjp(x, types, params, pairs, cot, lib=lib)
    return force_loss(F, Fstar), gx, ge, gs


def rollout_loss_grad(x0, v0, types, mass, params: Params, dt, nsteps, Fstar_end, lib=None):
    """L = mean |F(x_N) - F*|^2 after N steps, and its gradient w.r.t. x_0, v_0, eps, sigma."""
    lib = lib or load()
    xs, *_ = rollout(x0, v0, types, mass, params, dt, nsteps, record_masks=False, lib=lib)
    L, gxN, ge1, gs1 = force_loss_grad(xs[nsteps], types, params, Fstar_end, lib=lib)
    gx0, gv0, ge2, gs2 = rollout_vjp(x0, v0, types, mass, params, dt, nsteps, gxN, np.zeros_like(gxN), lib=lib)
    return L, gx0, gv0, ge1 + ge2, gs1 + gs2


def thermostat(v, types, mass, params: Params, target, max_change, lib=None):
    """Velocity scaling towards the target temperature by at most max_change
    (walled heating sphere, Sec. 6).  Returns (scaled v, T before)."""
    lib = lib or load()
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3).copy()
    n = v.shape[0]
    types = np.zeros(n, np.int32) if types is None else np.ascontiguousarray(types, np.int32)
    mass = np.ascontiguousarray(np.atleast_1d(np.asarray(mass, np.float64)))
    T = lib.orc_thermostat(n, _dp(v), _ip(types), _dp(mass), ctypes.byref(params), float(target), float(max_change))
    return v, T
