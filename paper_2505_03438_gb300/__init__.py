"""Python binding of libljsel, the GB300 library for short-range LJ molecular
dynamics with run-time configuration selection (arXiv 2505.03438).

Argument marshalling only: every step of the method runs in the CUDA library
behind the C ABI of ``include/ljsel.h``.  The functions below carry the same
names as the C entry points.  Arrays may be numpy arrays (host) or torch
tensors (host or CUDA); torch is used only for device memory and streams.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2505_03438_gb300.build``); importing a function when the
shared library is missing raises RuntimeError -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LJSEL_LIBRARY=checked selects the bounds-checked build (see build.py)
LIB_PATH = os.path.join(_HERE, "_build", "libljsel_checked.so" if os.environ.get("LJSEL_LIBRARY") == "checked"
                        else "libljsel.so")
MAX_TYPES = 4

METHOD_LC, METHOD_VL, METHOD_CLUSTER, METHOD_VLW = 0, 1, 2, 3
METHOD_NAMES = {METHOD_LC: "LC", METHOD_VL: "VL", METHOD_CLUSTER: "CL", METHOD_VLW: "VLW"}

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_CAPACITY", 5: "ERR_BOX",
          6: "ERR_NONFINITE", 7: "ERR_TIMEOUT", 8: "ERR_STATE", 9: "ERR_UNSUPPORTED"}


class LjselError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class ljsel_params(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("ntypes", ctypes.c_int32),
        ("shift_potential", ctypes.c_int32),
        ("eps", ctypes.c_double * (MAX_TYPES * MAX_TYPES)),
        ("sigma", ctypes.c_double * (MAX_TYPES * MAX_TYPES)),
        ("rcut", ctypes.c_double * (MAX_TYPES * MAX_TYPES)),
        ("mass", ctypes.c_double * MAX_TYPES),
        ("skin", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("use_graphs", ctypes.c_int32),
        ("walls", ctypes.c_int32 * 3),
        ("pad", ctypes.c_int32),
    ]


class ljsel_config(ctypes.Structure):
    _fields_ = [
        ("method", ctypes.c_int32),
        ("cluster_size", ctypes.c_int32),
        ("newton3", ctypes.c_int32),
        ("threads_per_unit", ctypes.c_int32),
        ("rebuild_interval", ctypes.c_int32),
        ("csf", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

    def name(self):
        m = METHOD_NAMES[self.method]
        if self.method == METHOD_CLUSTER:
            m += "%d" % self.cluster_size
        return "%s-%s-t%d-R%d-csf%g" % (m, "N3L" if self.newton3 else "noN3L", self.threads_per_unit,
                                         self.rebuild_interval, self.csf)


def config_from_name(name):
    """The configuration a name of ljsel_config.name() denotes, e.g.
    'VL-noN3L-t2-R10-csf1' or 'CL8-N3L-t8-R10-csf1'."""
    import re
    m = re.match(r"^(LC|VLW|VL|CL)(\d+)?-(N3L|noN3L)-t(\d+)-R(\d+)-csf([0-9.]+)$", name)
    if not m:
        raise ValueError("not a configuration name: %r" % name)
    meth, M, n3, t, R, csf = m.groups()
    return make_config(meth, cluster_size=int(M) if M else 1, newton3=(n3 == "N3L"), threads_per_unit=int(t),
                       rebuild_interval=int(R), csf=float(csf))


class ljsel_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("mean", "rel_std", "median", "max", "nbins", "nempty", "skin",
                                                "threads")]


class ljsel_counters(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("steps", "rebuilds", "early_rebuilds", "list_entries",
                                               "list_capacity", "nclusters", "ncells", "capacity_retries",
                                               "replica_rebuilds", "longest_row")]


class ljsel_tuner_opts(ctypes.Structure):
    _fields_ = [
        ("strategy", ctypes.c_int32),
        ("trial_steps", ctypes.c_int32),
        ("predict_factor", ctypes.c_double),
        ("blacklist_factor", ctypes.c_double),
        ("retrial_phases", ctypes.c_int32),
        ("ncandidates", ctypes.c_int32),
        ("candidates", ctypes.POINTER(ljsel_config)),
        ("probe_steps", ctypes.c_int32),
        ("forest_top", ctypes.c_int32),
        ("probe_factor", ctypes.c_double),
        ("skip_within", ctypes.c_double),
    ]


class ljsel_forest(ctypes.Structure):
    _fields_ = [
        ("ntrees", ctypes.c_int32),
        ("nclasses", ctypes.c_int32),
        ("nfeatures", ctypes.c_int32),
        ("nnodes", ctypes.c_int32),
        ("root", ctypes.c_void_p),
        ("feature", ctypes.c_void_p),
        ("threshold", ctypes.c_void_p),
        ("left", ctypes.c_void_p),
        ("right", ctypes.c_void_p),
        ("value", ctypes.c_void_p),
        ("classes", ctypes.POINTER(ljsel_config)),
    ]


class ljsel_tuner_report(ctypes.Structure):
    _fields_ = [
        ("phase", ctypes.c_int32),
        ("ntrialled", ctypes.c_int32),
        ("nblacklisted", ctypes.c_int32),
        ("chosen_index", ctypes.c_int32),
        ("chosen_cost_ms", ctypes.c_double),
        ("phase_ms", ctypes.c_double),
        ("overhead_ms", ctypes.c_double),
        ("trial_steps_total", ctypes.c_int64),
        ("nprobed_out", ctypes.c_int32),
        ("skipped", ctypes.c_int32),
        ("expert_input", ctypes.c_double),
        ("rebuild_every", ctypes.c_double),
    ]


class ljsel_profile(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("rebuilds", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("rebuild_ms", ctypes.c_double), ("force_ms", ctypes.c_double), ("update_ms", ctypes.c_double),
                ("control_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


class ljsel_batch_tile(ctypes.Structure):
    _fields_ = [("threads_per_particle", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("persistent_ctas_per_sm", ctypes.c_int32), ("rebuild_interval", ctypes.c_int32)]

    def as_tuple(self):
        return (self.threads_per_particle, self.block_threads, self.persistent_ctas_per_sm, self.rebuild_interval)


class ljsel_peaks(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("fp32_tflops", "fp32x2_tflops", "fp64_tflops", "rcp_tops")]


_P = ctypes.c_void_p
_SIGS = {
    "ljsel_last_error": ([], ctypes.c_char_p),
    "ljsel_abi_version": ([], ctypes.c_int32),
    "ljsel_selftest_wait_timeout": ([ctypes.c_int64], ctypes.c_int),
    "ljsel_create": ([ctypes.POINTER(ljsel_params), ctypes.c_int64, _P, _P, _P, ctypes.c_int32, _P,
                      ctypes.POINTER(_P)], ctypes.c_int),
    "ljsel_destroy": ([_P], ctypes.c_int),
    "ljsel_set_config": ([_P, ctypes.POINTER(ljsel_config)], ctypes.c_int),
    "ljsel_get_config": ([_P, ctypes.POINTER(ljsel_config)], ctypes.c_int),
    "ljsel_rebuild": ([_P], ctypes.c_int),
    "ljsel_compute": ([_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                      ctypes.c_int),
    "ljsel_step": ([_P, ctypes.c_int64], ctypes.c_int),
    "ljsel_thermostat": ([_P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ljsel_get_state": ([_P, _P, _P, ctypes.c_int32], ctypes.c_int),
    "ljsel_set_state": ([_P, _P, _P, ctypes.c_int32], ctypes.c_int),
    "ljsel_get_work_positions": ([_P, _P, ctypes.c_int32], ctypes.c_int),
    "ljsel_move_particles": ([_P, _P, ctypes.c_int32], ctypes.c_int),
    "ljsel_get_pairs": ([_P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "ljsel_get_energy": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ljsel_get_stats": ([_P, ctypes.POINTER(ljsel_stats)], ctypes.c_int),
    "ljsel_get_counters": ([_P, ctypes.POINTER(ljsel_counters)], ctypes.c_int),
    "ljsel_autotune": ([_P, ctypes.POINTER(ljsel_tuner_opts), ctypes.POINTER(ljsel_config),
                        ctypes.POINTER(ljsel_tuner_report)], ctypes.c_int),
    "ljsel_compute_forces_noalloc": ([ctypes.POINTER(ljsel_params), ctypes.c_int64, _P, _P, _P,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _P],
                                     ctypes.c_int),
    "ljsel_profile_steps": ([_P, ctypes.c_int64, ctypes.POINTER(ljsel_profile)], ctypes.c_int),
    "ljsel_default_candidates": ([_P, ctypes.c_int32, ctypes.POINTER(ljsel_config), ctypes.POINTER(ctypes.c_int32)],
                                 ctypes.c_int),
    "ljsel_set_pair_params": ([_P, _P, _P, _P], ctypes.c_int),
    "ljsel_force_vjp": ([_P, _P, ctypes.c_int32, _P, _P, _P], ctypes.c_int),
    "ljsel_rollout": ([_P, ctypes.c_int64, ctypes.c_int64], ctypes.c_int),
    "ljsel_rollout_vjp": ([_P, _P, _P, ctypes.c_int32, _P, _P, _P, _P], ctypes.c_int),
    "ljsel_batch_create": ([ctypes.POINTER(ljsel_params), ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32, _P,
                            ctypes.POINTER(_P)], ctypes.c_int),
    "ljsel_batch_destroy": ([_P], ctypes.c_int),
    "ljsel_batch_set_tile": ([_P, ctypes.POINTER(ljsel_batch_tile)], ctypes.c_int),
    "ljsel_batch_get_tile": ([_P, ctypes.POINTER(ljsel_batch_tile)], ctypes.c_int),
    "ljsel_batch_step": ([_P, ctypes.c_int64], ctypes.c_int),
    "ljsel_batch_step_eager": ([_P, ctypes.c_int64], ctypes.c_int),
    "ljsel_batch_compute": ([_P, _P, ctypes.c_int32, _P, _P], ctypes.c_int),
    "ljsel_batch_get_state": ([_P, _P, _P, ctypes.c_int32], ctypes.c_int),
    "ljsel_batch_get_work_positions": ([_P, _P], ctypes.c_int),
    "ljsel_batch_get_pairs": ([_P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "ljsel_batch_get_counters": ([_P, ctypes.POINTER(ljsel_counters)], ctypes.c_int),
    "ljsel_batch_profile_steps": ([_P, ctypes.c_int64, ctypes.POINTER(ljsel_profile)], ctypes.c_int),
    "ljsel_batch_autotune": ([_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.POINTER(ljsel_batch_tile), _P],
                             ctypes.c_int),
    "ljsel_predictive_trials": ([ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_double,
                                 ctypes.c_int32, _P], ctypes.c_int),
    "ljsel_forest_predict": ([ctypes.POINTER(ljsel_forest), _P, _P], ctypes.c_int),
    "ljsel_set_forest": ([_P, ctypes.POINTER(ljsel_forest)], ctypes.c_int),
    "ljsel_tuner_costs": ([_P, ctypes.c_int32, ctypes.POINTER(ljsel_config), _P, _P, ctypes.POINTER(ctypes.c_int32)],
                          ctypes.c_int),
    "ljsel_measure_peaks": ([ctypes.c_double, ctypes.POINTER(ljsel_peaks)], ctypes.c_int),
    "ljsel_set_list_capacity": ([_P, ctypes.c_int64], ctypes.c_int),
    "ljsel_batch_set_list_capacity": ([_P, ctypes.c_int64], ctypes.c_int),
    "ljsel_expert_suitability": ([ctypes.POINTER(ljsel_config), ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
                                 ctypes.c_int),
}
EXPORTED = tuple(_SIGS)
_lib = None


def lib():
    """Load libljsel.so (raises RuntimeError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libljsel.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        raise LjselError(st, lib().ljsel_last_error().decode())


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (C-contiguous)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def make_params(box, eps=1.0, sigma=1.0, rcut=2.5, mass=1.0, skin=0.3, dt=0.005, shift=True, precision=0,
                use_graphs=True, walls=(0, 0, 0)) -> ljsel_params:
    eps = np.atleast_2d(np.asarray(eps, np.float64))
    sigma = np.atleast_2d(np.asarray(sigma, np.float64))
    nt = eps.shape[0]
    rcut = np.asarray(rcut, np.float64)
    if rcut.ndim == 0:
        rcut = np.full((nt, nt), float(rcut))
    mass = np.broadcast_to(np.asarray(mass, np.float64), (nt,))
    p = ljsel_params()
    box = np.broadcast_to(np.asarray(box, np.float64), (3,))
    for d in range(3):
        p.box[d] = float(box[d])
    p.ntypes = nt
    p.shift_potential = 1 if shift else 0
    for a in range(nt):
        p.mass[a] = float(mass[a])
        for b in range(nt):
            p.eps[a * nt + b] = float(eps[a, b])
            p.sigma[a * nt + b] = float(sigma[a, b])
            p.rcut[a * nt + b] = float(rcut[a, b])
    p.skin = float(skin)
    p.dt = float(dt)
    p.precision = int(precision)
    p.use_graphs = 1 if use_graphs else 0
    for d in range(3):
        p.walls[d] = 1 if walls[d] else 0
    return p


def make_config(method="VL", cluster_size=1, newton3=False, threads_per_unit=1, rebuild_interval=10, csf=1.0):
    c = ljsel_config()
    c.method = {"LC": METHOD_LC, "VL": METHOD_VL, "CL": METHOD_CLUSTER, "CLUSTER": METHOD_CLUSTER,
                "VLW": METHOD_VLW}.get(method, method)
    c.cluster_size = int(cluster_size)
    c.newton3 = 1 if newton3 else 0
    c.threads_per_unit = int(threads_per_unit)
    c.rebuild_interval = int(rebuild_interval)
    c.csf = float(csf)
    return c


# --- the C entry points, same names ------------------------------------------

def ljsel_last_error() -> str:
    return lib().ljsel_last_error().decode()


def ljsel_abi_version() -> int:
    return int(lib().ljsel_abi_version())


def ljsel_selftest_wait_timeout(polls=1 << 16):
    """Runs the bounded-wait failure path on the GPU; returns the status code (LJSEL_ERR_TIMEOUT expected)."""
    return int(lib().ljsel_selftest_wait_timeout(int(polls)))


def ljsel_create(params: ljsel_params, n, pos, vel, types=None, stream=None):
    pp, dev = _ptr(pos)
    vp, dv = _ptr(vel)
    tp, dt = _ptr(types)
    if not (dev == dv and (types is None or dt == dev)):
        raise ValueError("pos, vel and types must all be host or all be device arrays")
    h = ctypes.c_void_p()
    _check(lib().ljsel_create(ctypes.byref(params), int(n), pp, vp, tp, dev, stream, ctypes.byref(h)))
    return h


def ljsel_destroy(h):
    _check(lib().ljsel_destroy(h))


def ljsel_set_config(h, cfg: ljsel_config):
    _check(lib().ljsel_set_config(h, ctypes.byref(cfg)))


def ljsel_get_config(h) -> ljsel_config:
    c = ljsel_config()
    _check(lib().ljsel_get_config(h, ctypes.byref(c)))
    return c


def ljsel_rebuild(h):
    _check(lib().ljsel_rebuild(h))


def ljsel_compute(h, forces=None, sums=True):
    """Forces (into `forces`) and, with sums=True, (energy, virial); with
    sums=False only the forces, by the stepping kernels' arithmetic."""
    e = ctypes.c_double()
    w = ctypes.c_double()
    fp, dev = _ptr(forces)
    if sums:
        _check(lib().ljsel_compute(h, fp, dev, ctypes.byref(e), ctypes.byref(w)))
        return e.value, w.value
    _check(lib().ljsel_compute(h, fp, dev, None, None))
    return None


def ljsel_step(h, nsteps):
    _check(lib().ljsel_step(h, int(nsteps)))


def ljsel_thermostat(h, target, max_change):
    """Velocity scaling towards `target` by at most `max_change`; returns T before."""
    t = ctypes.c_double()
    _check(lib().ljsel_thermostat(h, float(target), float(max_change), ctypes.byref(t)))
    return t.value


def ljsel_get_state(h, pos=None, vel=None):
    pp, d1 = _ptr(pos)
    vp, d2 = _ptr(vel)
    if pos is not None and vel is not None and d1 != d2:
        raise ValueError("pos and vel must be both host or both device")
    _check(lib().ljsel_get_state(h, pp, vp, d1 if pos is not None else d2))


def ljsel_set_state(h, pos=None, vel=None):
    pp, d1 = _ptr(pos)
    vp, d2 = _ptr(vel)
    if pos is not None and vel is not None and d1 != d2:
        raise ValueError("pos and vel must be both host or both device")
    _check(lib().ljsel_set_state(h, pp, vp, d1 if pos is not None else d2))


def ljsel_move_particles(h, pos):
    p, d = _ptr(pos)
    _check(lib().ljsel_move_particles(h, p, d))


def ljsel_get_work_positions(h, pos):
    p, d = _ptr(pos)
    _check(lib().ljsel_get_work_positions(h, p, d))


def ljsel_get_pairs(h, cap):
    buf = np.zeros((max(int(cap), 1), 2), np.int32)
    cnt = ctypes.c_int64()
    _check(lib().ljsel_get_pairs(h, int(cap), buf.ctypes.data, ctypes.byref(cnt)))
    return buf[:min(cnt.value, int(cap))], cnt.value


def ljsel_get_energy(h):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().ljsel_get_energy(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def ljsel_get_stats(h) -> dict:
    s = ljsel_stats()
    _check(lib().ljsel_get_stats(h, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in s._fields_}


def ljsel_get_counters(h) -> dict:
    c = ljsel_counters()
    _check(lib().ljsel_get_counters(h, ctypes.byref(c)))
    return {k: getattr(c, k) for k, _ in c._fields_}


def ljsel_profile_steps(h, nsteps) -> dict:
    p = ljsel_profile()
    _check(lib().ljsel_profile_steps(h, int(nsteps), ctypes.byref(p)))
    return {k: getattr(p, k) for k, _ in p._fields_}


def ljsel_compute_forces_noalloc(params: ljsel_params, n, pos, forces, types=None, stream=None):
    """Allocation-free force evaluation (device pos/types/forces); returns (energy, virial)."""
    pp, d1 = _ptr(pos)
    fp, d2 = _ptr(forces)
    tp, d3 = _ptr(types)
    if not (d1 and d2 and (types is None or d3)):
        raise ValueError("pos, forces and types must be device tensors")
    e = ctypes.c_double()
    w = ctypes.c_double()
    _check(lib().ljsel_compute_forces_noalloc(ctypes.byref(params), int(n), pp, tp, fp, ctypes.byref(e),
                                              ctypes.byref(w), stream))
    return e.value, w.value


def ljsel_set_list_capacity(h, entries):
    _check(lib().ljsel_set_list_capacity(h, int(entries)))


def ljsel_batch_set_list_capacity(b, entries):
    _check(lib().ljsel_batch_set_list_capacity(b, int(entries)))


def ljsel_expert_suitability(cfg: ljsel_config, mean_per_bin) -> float:
    """The Expert strategy's rating of a configuration (host only)."""
    out = ctypes.c_double()
    _check(lib().ljsel_expert_suitability(ctypes.byref(cfg), ctypes.c_double(mean_per_bin), ctypes.byref(out)))
    return out.value


def ljsel_measure_peaks(target_ms=30.0) -> dict:
    """Measured FP32 / packed FP32x2 / FP64 fused multiply-add rates (TFLOP/s)
    and the FP32 reciprocal rate (Tops/s) of the current device."""
    p = ljsel_peaks()
    _check(lib().ljsel_measure_peaks(ctypes.c_double(target_ms), ctypes.byref(p)))
    return {k: getattr(p, k) for k, _ in p._fields_}


def ljsel_default_candidates(h):
    cnt = ctypes.c_int32()
    _check(lib().ljsel_default_candidates(h, 0, None, ctypes.byref(cnt)))
    arr = (ljsel_config * max(cnt.value, 1))()
    _check(lib().ljsel_default_candidates(h, cnt.value, arr, ctypes.byref(cnt)))
    return [arr[k] for k in range(cnt.value)]


def ljsel_autotune(h, strategy=0, trial_steps=10, predict_factor=2.0, blacklist_factor=10.0, retrial_phases=4,
                   candidates=None, probe_steps=0, probe_factor=2.0, skip_within=0.0, forest_top=1):
    o = ljsel_tuner_opts()
    o.skip_within = float(skip_within)
    o.forest_top = int(forest_top)
    o.strategy = {"full": 0, "predictive": 1, "expert": 2, "forest": 3}.get(strategy, strategy)
    o.probe_steps = int(probe_steps)
    o.probe_factor = float(probe_factor)
    o.trial_steps = int(trial_steps)
    o.predict_factor = float(predict_factor)
    o.blacklist_factor = float(blacklist_factor)
    o.retrial_phases = int(retrial_phases)
    arr = None
    if candidates:
        arr = (ljsel_config * len(candidates))(*candidates)
        o.ncandidates = len(candidates)
        o.candidates = arr
    chosen = ljsel_config()
    rep = ljsel_tuner_report()
    _check(lib().ljsel_autotune(h, ctypes.byref(o), ctypes.byref(chosen), ctypes.byref(rep)))
    return chosen, {k: getattr(rep, k) for k, _ in rep._fields_}


def ljsel_predictive_trials(phase, history, last_trial_phase, blacklisted, incumbent=-1, predict_factor=2.0,
                            retrial_phases=4):
    """Trial set of one Predictive tuning phase (host only).  history[k] is a
    list of (phase, cost) measurements of configuration k, oldest first (the
    last two are used).  Returns a list of 0/1 per configuration."""
    n = len(history)
    hn = np.zeros(n, np.int32)
    hp = np.zeros(2 * n, np.int32)
    hc = np.zeros(2 * n, np.float64)
    for k, hs in enumerate(history):
        hs = list(hs)[-2:]
        hn[k] = len(hs)
        for q, (ph, c) in enumerate(hs):
            slot = 2 * k + (1 if len(hs) == 1 else q)
            hp[slot], hc[slot] = ph, c
    lt = np.ascontiguousarray(last_trial_phase, np.int32)
    bl = np.ascontiguousarray(blacklisted, np.int32)
    out = np.zeros(max(n, 1), np.int32)
    _check(lib().ljsel_predictive_trials(n, int(phase), hn.ctypes.data, hp.ctypes.data, hc.ctypes.data, lt.ctypes.data,
                                         bl.ctypes.data, int(incumbent), float(predict_factor), int(retrial_phases),
                                         out.ctypes.data))
    return out[:n].tolist()


_FOREST_STRUCTS = {}


def _forest_struct(model):
    """ljsel_forest over the arrays of a forest model (dict of numpy arrays,
    see paper_2505_03438_gb300.forest); the arrays are kept alive on the
    returned struct.  The struct of a model object is built once (turning a
    loaded model's lists into arrays takes longer than a short run's steps)
    and rebuilt when one of its arrays is replaced."""
    key = id(model)
    ids = tuple(id(model[k]) for k in ("root", "feature", "threshold", "left", "right", "value", "classes"))
    hit = _FOREST_STRUCTS.get(key)
    if hit is not None and hit[0] is model and hit[1] == ids:
        return hit[2]
    keep = {
        "root": np.ascontiguousarray(model["root"], np.int32),
        "feature": np.ascontiguousarray(model["feature"], np.int32),
        "threshold": np.ascontiguousarray(model["threshold"], np.float64),
        "left": np.ascontiguousarray(model["left"], np.int32),
        "right": np.ascontiguousarray(model["right"], np.int32),
        "value": np.ascontiguousarray(model["value"], np.float64),
    }
    names = list(model["classes"])
    cls = (ljsel_config * max(len(names), 1))(*[config_from_name(c) for c in names])
    f = ljsel_forest()
    f.ntrees = len(keep["root"])
    f.nclasses = len(names)
    f.nfeatures = int(model["nfeatures"])
    f.nnodes = len(keep["feature"])
    for k, a in keep.items():
        setattr(f, k, a.ctypes.data)
    f.classes = cls
    f._keep = (keep, cls)
    if len(_FOREST_STRUCTS) > 8:
        _FOREST_STRUCTS.clear()
    _FOREST_STRUCTS[key] = (model, ids, f)
    return f


def ljsel_forest_predict(model, x):
    """Class probabilities of a forest model for one feature vector (host)."""
    f = _forest_struct(model)
    xv = np.ascontiguousarray(x, np.float64)
    out = np.zeros(max(f.nclasses, 1))
    _check(lib().ljsel_forest_predict(ctypes.byref(f), xv.ctypes.data, out.ctypes.data))
    return out[:f.nclasses]


def ljsel_set_forest(h, model):
    f = _forest_struct(model)
    _check(lib().ljsel_set_forest(h, ctypes.byref(f)))


def ljsel_tuner_costs(h):
    """{configuration name: (cost ms per step, phase)} of every configuration
    trialled so far, from its most recent trial."""
    cnt = ctypes.c_int32()
    _check(lib().ljsel_tuner_costs(h, 0, None, None, None, ctypes.byref(cnt)))
    n = cnt.value
    cfgs = (ljsel_config * max(n, 1))()
    cost = np.zeros(max(n, 1))
    ph = np.zeros(max(n, 1), np.int32)
    _check(lib().ljsel_tuner_costs(h, n, cfgs, cost.ctypes.data, ph.ctypes.data, ctypes.byref(cnt)))
    return {cfgs[k].name(): (float(cost[k]), int(ph[k])) for k in range(n)}


def _table(a, nt):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), (nt, nt)))
    return a


def ljsel_set_pair_params(h, eps, sigma, rcut=None):
    """Replace the ntypes x ntypes eps/sigma (and optionally rcut) tables."""
    eps = np.ascontiguousarray(np.atleast_2d(np.asarray(eps, np.float64)))
    nt = eps.shape[0]
    sigma = _table(sigma, nt)
    rc = None if rcut is None else _table(rcut, nt)
    _check(lib().ljsel_set_pair_params(h, eps.ctypes.data, sigma.ctypes.data, None if rc is None else rc.ctypes.data))


def ljsel_force_vjp(h, cot, g_pos=None, ntypes=1):
    """(dF/dx)^T cot into g_pos (same residency as cot); returns (g_eps, g_sigma) as ntypes x ntypes arrays."""
    cp, d1 = _ptr(cot)
    gp, d2 = _ptr(g_pos)
    if g_pos is not None and d1 != d2:
        raise ValueError("cot and g_pos must be both host or both device")
    ge = np.zeros((ntypes, ntypes))
    gs = np.zeros((ntypes, ntypes))
    _check(lib().ljsel_force_vjp(h, cp, d1, gp, ge.ctypes.data, gs.ctypes.data))
    return ge, gs


def ljsel_rollout(h, nsteps, every):
    _check(lib().ljsel_rollout(h, int(nsteps), int(every)))


def ljsel_rollout_vjp(h, xbar, vbar=None, g_x0=None, g_v0=None, ntypes=1):
    """Cotangents of (x_0, v_0) into g_x0/g_v0 (same residency as xbar); returns (g_eps, g_sigma)."""
    xp, d = _ptr(xbar)
    for a in (vbar, g_x0, g_v0):
        if a is not None and _ptr(a)[1] != d:
            raise ValueError("xbar, vbar, g_x0 and g_v0 must share one residency")
    ge = np.zeros((ntypes, ntypes))
    gs = np.zeros((ntypes, ntypes))
    _check(lib().ljsel_rollout_vjp(h, xp, _ptr(vbar)[0], d, _ptr(g_x0)[0], _ptr(g_v0)[0], ge.ctypes.data,
                                   gs.ctypes.data))
    return ge, gs


class System:
    """Owner of one ljsel handle (destroyed with the object); marshalling only."""

    def __init__(self, scenario=None, *, x=None, v=None, types=None, box=None, eps=None, sigma=None, rcut=None,
                 mass=None, skin=None, dt=None, shift=None, precision=0, use_graphs=True, stream=None, walls=None):
        sc = dict(scenario or {})
        pick = lambda val, key, default: val if val is not None else sc.get(key, default)
        x, v, types = pick(x, "x", None), pick(v, "v", None), pick(types, "types", None)
        box = pick(box, "box", None)
        self.params = make_params(box, pick(eps, "eps", 1.0), pick(sigma, "sigma", 1.0), pick(rcut, "rcut", 2.5),
                                  pick(mass, "mass", 1.0), pick(skin, "skin", 0.3), pick(dt, "dt", 0.005),
                                  pick(shift, "shift", True), precision, use_graphs,
                                  pick(walls, "walls", (0, 0, 0)))
        x = np.ascontiguousarray(x, np.float64) if isinstance(x, np.ndarray) else x
        v = np.ascontiguousarray(v, np.float64) if isinstance(v, np.ndarray) else v
        if isinstance(types, np.ndarray):
            types = np.ascontiguousarray(types, np.int32)
        self.n = int(x.shape[0])
        self.types = None if types is None else (types if isinstance(types, np.ndarray) else types.cpu().numpy())
        self.h = ljsel_create(self.params, self.n, x, v, types, stream)

    def close(self):
        if getattr(self, "h", None):
            ljsel_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, cfg=None, **kw):
        ljsel_set_config(self.h, cfg if cfg is not None else make_config(**kw))
        self._rollout_valid = False

    def config(self):
        return ljsel_get_config(self.h)

    def compute(self):
        F = np.zeros((self.n, 3))
        e, w = ljsel_compute(self.h, F)
        return F, e, w

    def forces(self):
        """Forces only (n x 3), by the force arithmetic of the stepping kernels."""
        F = np.zeros((self.n, 3))
        ljsel_compute(self.h, F, sums=False)
        return F

    def step(self, nsteps):
        ljsel_step(self.h, nsteps)

    def thermostat(self, target, max_change):
        return ljsel_thermostat(self.h, target, max_change)

    def state(self):
        x = np.zeros((self.n, 3))
        v = np.zeros((self.n, 3))
        ljsel_get_state(self.h, x, v)
        return x, v

    def set_state(self, x, v):
        ljsel_set_state(self.h, np.ascontiguousarray(x, np.float64), np.ascontiguousarray(v, np.float64))

    def work_positions(self):
        x = np.zeros((self.n, 3))
        ljsel_get_work_positions(self.h, x)
        return x

    def move_particles(self, x):
        ljsel_move_particles(self.h, np.ascontiguousarray(x, np.float64))

    def pairs(self, cap=None):
        if cap is None:
            _, cnt = ljsel_get_pairs(self.h, 0)
            cap = cnt
        p, cnt = ljsel_get_pairs(self.h, cap)
        return p, cnt

    def energy(self):
        return ljsel_get_energy(self.h)

    def stats(self):
        return ljsel_get_stats(self.h)

    def set_forest(self, model=None):
        """Install a random-forest model (a dict of paper_2505_03438_gb300.forest;
        None: the model shipped with the package) for autotune(strategy="forest")."""
        if model is None:
            from . import forest
            model = forest.load()
        ljsel_set_forest(self.h, model)

    def counters(self):
        return ljsel_get_counters(self.h)

    def profile(self, nsteps):
        return ljsel_profile_steps(self.h, nsteps)

    def autotune(self, **kw):
        return ljsel_autotune(self.h, **kw)

    def rebuild(self):
        ljsel_rebuild(self.h)

    def checkpoint(self, path):
        """Positions (wrapped), integer-step velocities, types, parameters and the
        configuration to an .npz file; System.from_checkpoint resumes from it."""
        x, v = self.state()
        t = np.zeros(self.n, np.int32) if self.types is None else np.asarray(self.types, np.int32)
        np.savez(path, x=x, v=v, types=t, params=np.frombuffer(bytes(self.params), np.uint8),
                 config=np.frombuffer(bytes(self.config()), np.uint8))

    @classmethod
    def from_checkpoint(cls, path, stream=None):
        z = np.load(path)
        obj = cls.__new__(cls)
        obj.params = ljsel_params.from_buffer_copy(z["params"].tobytes())
        obj.n = int(z["x"].shape[0])
        obj.types = np.ascontiguousarray(z["types"], np.int32)
        obj.h = ljsel_create(obj.params, obj.n, np.ascontiguousarray(z["x"]), np.ascontiguousarray(z["v"]),
                             obj.types, stream)
        ljsel_set_config(obj.h, ljsel_config.from_buffer_copy(z["config"].tobytes()))
        return obj

    @property
    def ntypes(self):
        return int(self.params.ntypes)

    def set_pair_params(self, eps, sigma, rcut=None):
        nt = self.ntypes
        tab = lambda a: np.broadcast_to(np.asarray(a, np.float64), (nt, nt)).reshape(-1)
        new = [(self.params.eps, tab(eps)), (self.params.sigma, tab(sigma))]
        if rcut is not None:
            new.append((self.params.rcut, tab(rcut)))
        ljsel_set_pair_params(self.h, eps, sigma, rcut)
        changed = False
        for dst, src in new:
            for k in range(nt * nt):
                changed |= dst[k] != float(src[k])
                dst[k] = float(src[k])
        if changed:
            self._rollout_valid = False  # the library dropped its rollout record

    def has_rollout(self):
        return getattr(self, "_rollout_valid", False)

    def force_vjp(self, cot):
        """Returns (g_pos, g_eps, g_sigma) for a host cotangent (n x 3)."""
        g = np.zeros((self.n, 3))
        ge, gs = ljsel_force_vjp(self.h, np.ascontiguousarray(cot, np.float64), g, self.ntypes)
        return g, ge, gs

    def rollout(self, nsteps, every):
        ljsel_rollout(self.h, nsteps, every)
        self._rollout_valid = True

    def rollout_vjp(self, xbar, vbar=None):
        """Returns (g_x0, g_v0, g_eps, g_sigma) for host cotangents of the final state."""
        gx = np.zeros((self.n, 3))
        gv = np.zeros((self.n, 3))
        vb = None if vbar is None else np.ascontiguousarray(vbar, np.float64)
        ge, gs = ljsel_rollout_vjp(self.h, np.ascontiguousarray(xbar, np.float64), vb, gx, gv, self.ntypes)
        return gx, gv, ge, gs


# --- batched replicas -----------------------------------------------------------

def ljsel_batch_create(params: ljsel_params, boxes, counts, pos, vel, stream=None):
    boxes = np.ascontiguousarray(boxes, np.float64).reshape(-1, 3)
    counts = np.ascontiguousarray(counts, np.int64)
    pp, d1 = _ptr(pos)
    vp, d2 = _ptr(vel)
    if d1 != d2:
        raise ValueError("pos and vel must be both host or both device")
    h = ctypes.c_void_p()
    _check(lib().ljsel_batch_create(ctypes.byref(params), len(counts), boxes.ctypes.data, counts.ctypes.data, pp, vp,
                                    d1, stream, ctypes.byref(h)))
    return h


def ljsel_batch_destroy(b):
    _check(lib().ljsel_batch_destroy(b))


def make_tile(threads_per_particle=1, block_threads=128, persistent_ctas_per_sm=0, rebuild_interval=10):
    return ljsel_batch_tile(int(threads_per_particle), int(block_threads), int(persistent_ctas_per_sm),
                            int(rebuild_interval))


def ljsel_batch_set_tile(b, tile: ljsel_batch_tile):
    _check(lib().ljsel_batch_set_tile(b, ctypes.byref(tile)))


def ljsel_batch_get_tile(b) -> ljsel_batch_tile:
    t = ljsel_batch_tile()
    _check(lib().ljsel_batch_get_tile(b, ctypes.byref(t)))
    return t


def ljsel_batch_step(b, nsteps):
    _check(lib().ljsel_batch_step(b, int(nsteps)))


def ljsel_batch_step_eager(b, nsteps):
    _check(lib().ljsel_batch_step_eager(b, int(nsteps)))


def ljsel_batch_compute(b, forces=None, nrep=0):
    """Forces into ``forces`` (host or device); returns per-replica (energy, virial) arrays."""
    fp, d = _ptr(forces)
    e = np.zeros(max(nrep, 1))
    w = np.zeros(max(nrep, 1))
    _check(lib().ljsel_batch_compute(b, fp, d, e.ctypes.data if nrep else None, w.ctypes.data if nrep else None))
    return e[:nrep], w[:nrep]


def ljsel_batch_get_state(b, pos=None, vel=None):
    pp, d1 = _ptr(pos)
    vp, d2 = _ptr(vel)
    if pos is not None and vel is not None and d1 != d2:
        raise ValueError("pos and vel must be both host or both device")
    _check(lib().ljsel_batch_get_state(b, pp, vp, d1 if pos is not None else d2))


def ljsel_batch_get_work_positions(b, pos):
    p, d = _ptr(pos)
    if d:
        raise ValueError("work positions are returned to host memory")
    _check(lib().ljsel_batch_get_work_positions(b, p))


def ljsel_batch_get_pairs(b, cap):
    buf = np.zeros((max(int(cap), 1), 3), np.int32)
    cnt = ctypes.c_int64()
    _check(lib().ljsel_batch_get_pairs(b, int(cap), buf.ctypes.data, ctypes.byref(cnt)))
    return buf[:min(cnt.value, int(cap))], cnt.value


def ljsel_batch_get_counters(b) -> dict:
    c = ljsel_counters()
    _check(lib().ljsel_batch_get_counters(b, ctypes.byref(c)))
    return {k: getattr(c, k) for k, _ in c._fields_}


def ljsel_batch_profile_steps(b, nsteps) -> dict:
    p = ljsel_profile()
    _check(lib().ljsel_batch_profile_steps(b, int(nsteps), ctypes.byref(p)))
    return {k: getattr(p, k) for k, _ in p._fields_}


def ljsel_batch_autotune(b, trial_steps=20, candidates=None):
    """Full search over force-kernel tiles; returns (chosen tile, list of (tile, ms/step))."""
    n = len(candidates) if candidates else 0
    arr = (ljsel_batch_tile * max(n, 1))(*(candidates or []))
    costs = np.full(max(n, 10), -1.0)
    chosen = ljsel_batch_tile()
    _check(lib().ljsel_batch_autotune(b, int(trial_steps), n, arr if n else None, ctypes.byref(chosen),
                                      costs.ctypes.data))
    return chosen, costs[:max(n, 10)].tolist()


class Batch:
    """Owner of one ljsel batch handle; replicas given as a list of scenario dicts."""

    def __init__(self, replicas, precision=0, use_graphs=True, stream=None, device_inputs=None):
        r0 = replicas[0]
        self.counts = np.array([len(r["x"]) for r in replicas], np.int64)
        self.offsets = np.concatenate([[0], np.cumsum(self.counts)])
        self.nrep = len(replicas)
        self.ntot = int(self.counts.sum())
        boxes = np.stack([np.broadcast_to(np.asarray(r["box"], np.float64), (3,)) for r in replicas])
        self.boxes = boxes
        self.params = make_params(boxes[0], r0.get("eps", 1.0), r0.get("sigma", 1.0), r0.get("rcut", 2.5),
                                  r0.get("mass", 1.0), r0.get("skin", 0.3), r0.get("dt", 0.005), r0.get("shift", True),
                                  precision, use_graphs)
        x = np.ascontiguousarray(np.concatenate([r["x"] for r in replicas]), np.float64)
        v = np.ascontiguousarray(np.concatenate([r["v"] for r in replicas]), np.float64)
        if device_inputs is not None:
            x, v = device_inputs(x), device_inputs(v)
        self.h = ljsel_batch_create(self.params, boxes, self.counts, x, v, stream)

    def close(self):
        if getattr(self, "h", None):
            ljsel_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def split(self, a):
        return [a[self.offsets[r]:self.offsets[r + 1]] for r in range(self.nrep)]

    def step(self, nsteps, eager=False):
        (ljsel_batch_step_eager if eager else ljsel_batch_step)(self.h, nsteps)

    def compute(self):
        F = np.zeros((self.ntot, 3))
        e, w = ljsel_batch_compute(self.h, F, self.nrep)
        return F, e, w

    def state(self):
        x = np.zeros((self.ntot, 3))
        v = np.zeros((self.ntot, 3))
        ljsel_batch_get_state(self.h, x, v)
        return x, v

    def work_positions(self):
        x = np.zeros((self.ntot, 3))
        ljsel_batch_get_work_positions(self.h, x)
        return x

    def pairs(self):
        _, cnt = ljsel_batch_get_pairs(self.h, 0)
        p, cnt = ljsel_batch_get_pairs(self.h, cnt)
        return p

    def counters(self):
        return ljsel_batch_get_counters(self.h)

    def set_tile(self, **kw):
        ljsel_batch_set_tile(self.h, make_tile(**kw))

    def tile(self):
        return ljsel_batch_get_tile(self.h).as_tuple()

    def autotune(self, trial_steps=20, candidates=None):
        return ljsel_batch_autotune(self.h, trial_steps, candidates)

    def profile(self, nsteps):
        return ljsel_batch_profile_steps(self.h, nsteps)
