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
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)


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


def make_params(box, eps, sigma, rcut, shift=True) -> Params:
    """Pack a parameter set.  eps/sigma/rcut: scalars (one type) or ntypes x ntypes."""
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
