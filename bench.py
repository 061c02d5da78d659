#!/usr/bin/env python
"""Benchmark: LJ particle-steps/s on the homogeneous 1M-atom liquid, the
auto-tuned GPU path against every fixed configuration, with the roofline
fraction of the dominant kernel and of the whole step.

Workload (synthetic; the paper's md-flexible inputs are not available):
N = 1,048,576 LJ particles on a 64^3 x 4 fcc lattice, density 0.8442,
Maxwell-Boltzmann velocities at T = 0.72 (seed 2), cutoff 2.5 sigma with an
energy shift, skin 0.3 sigma, rebuild every 10 steps (or earlier when a
particle moves skin/2), dt 0.005, FP32 pair arithmetic with FP64
integration and sums.

A "step" is one Stormer-Verlet step of the whole system (binning, lists,
forces, update).  The timed region of the headline run holds one tuning
phase (with the default Random Forest strategy: the live statistics, the
forest's choice and the switch to it; trial steps of other strategies
advance the simulation and count as steps) followed by the remaining steps
with the chosen configuration.

Output: one compact JSON line (the last line printed); the per-leg details
(every fixed configuration, the other strategies, the batched, gradient and
heated-sphere legs) go to the file given by --details.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Multi-GPU: the path does not shard across GPUs here (one system per GPU);
--gpus N runs N independent replicas, one per rank, and reports the sum.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LJ particle-steps/s at 1M atoms, auto-tuned vs fixed config; % of roofline"
UNIT = "particle-steps/s"
WORKLOAD = "lj_liquid_1m: N=1048576 fcc 64^3x4, rho 0.8442, T 0.72, rc 2.5, skin 0.3, R 10"
# Algorithmic FP32 work per within-cutoff unordered pair with Newton's third
# law (FFMA = 2 flops): displacement 3, r^2 5, cutoff test 1, (sigma/r)^6 3,
# f/r 4, F_i 6, F_j 6.  The reciprocal runs on the MUFU pipe and is counted
# against its own peak.
FLOPS_PER_PAIR = 28
# Algorithmic per-particle figures of the other kernels of a step:
# the Stormer-Verlet update reads and writes the FP64 x, v (96 B), writes the
# FP32 working position (16 B) and reads the force (16 B), and issues 6 FP64
# instructions (3 adds for v, 3 fused multiply-adds for x; the FP32 <-> FP64
# conversions run on the integer pipes); a rebuild reads the working position and
# writes the sorted one and the permutation (36 B), 8 B per cell, reads the
# position once more for the lists (16 B) and writes 4 B per list entry.
UPDATE_BYTES_PER_PARTICLE = 128
UPDATE_FP64_PER_PARTICLE = 6
REBUILD_BYTES_PER_PARTICLE = 36 + 16
REBUILD_BYTES_PER_CELL = 8
LIST_BYTES_PER_ENTRY = 4
# DRAM bytes (read + write) of one launch of the force kernel (fused with the
# update when N3L is off) at N = 1,048,576, CSF 1, from ncu captures of those
# kernels; reported only when the chosen configuration is one of them.
FORCE_TRAFFIC_1M = {
    "VL-noN3L-t2": 491916288 + 57595648,
    "VL-N3L-t4": 340648192 + 15194368,
    "CL4-noN3L-t4": 283816960 + 19887360,
    "CL4-N3L-t8": 145644800 + 6951936,
}


def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time: every rank's figure, all-reduced with MAX."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n_per_rank, steps, ms):
    """Whole-job particle-steps/s of `world` independent replicas, each
    advancing n_per_rank particles `steps` steps, timed by the slowest rank."""
    return world * n_per_rank * steps / (ms * 1e-3)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons, started before
    the warm-up and stopped after the timed region (the timed region alone is
    often shorter than the sampling interval)."""

    def __init__(self, gpu_index, interval_ms=10):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", str(interval_ms)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
            time.sleep(0.3)  # the first sample takes a moment
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.05)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": "warm-up and timed region"}


def step_roofline(n, npairs, n3l, entries, ncell, rebuild_every, peaks, hbm_gbs):
    """Per-step roofline time T_roof = sum over the kernels of
    max(bytes / HBM bandwidth, operations / pipe peak), the rebuild amortised
    over the measured interval: the force kernel against the FP32 and MUFU
    peaks (algorithmic pairs only, N3L work), the update against HBM and
    FP64, the rebuild against HBM."""
    fp32 = max(peaks["fp32_tflops"], peaks["fp32x2_tflops"]) * 1e12
    t_force = max(npairs * FLOPS_PER_PAIR / fp32, npairs / (peaks["rcp_tops"] * 1e12))
    t_update = max(n * UPDATE_BYTES_PER_PARTICLE / (hbm_gbs * 1e9),
                   n * UPDATE_FP64_PER_PARTICLE / (peaks["fp64_tflops"] * 1e12 / 2.0))
    reb_bytes = n * REBUILD_BYTES_PER_PARTICLE + ncell * REBUILD_BYTES_PER_CELL + entries * LIST_BYTES_PER_ENTRY
    t_rebuild = reb_bytes / (hbm_gbs * 1e9)
    t = t_force + t_update + t_rebuild / max(rebuild_every, 1.0)
    return {"t_roof_us": 1e6 * t, "force_us": 1e6 * t_force, "update_us": 1e6 * t_update,
            "rebuild_us": 1e6 * t_rebuild, "rebuild_every": rebuild_every}


def oracle_rate(sc, budget_s=12.0, single=False):
    """The FP64 oracle (linked cells, OpenMP on all host cores) advancing a
    bounded number of Stormer-Verlet steps of the same system; with single,
    also one thread on a smaller sample of the same liquid."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    p = oracle.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], True)
    cell_min = 2.5 + sc["skin"]
    t0 = time.perf_counter()
    oracle.verlet_run(sc["x"], sc["v"], sc.get("types"), sc["mass"], p, sc["dt"], 1, cell_min=cell_min, nthreads=cores)
    t1 = time.perf_counter()
    per = (t1 - t0) / 2.0  # one call evaluates forces twice for one step
    nsteps = max(1, min(50, int(budget_s / max(per, 1e-3))))
    t0 = time.perf_counter()
    oracle.verlet_run(sc["x"], sc["v"], sc.get("types"), sc["mass"], p, sc["dt"], nsteps, cell_min=cell_min,
                      nthreads=cores)
    t1 = time.perf_counter()
    n = len(sc["x"])
    out = {"value": n * nsteps / (t1 - t0), "unit": UNIT, "cores": cores, "kind": "oracle", "steps": nsteps,
           "seconds": t1 - t0,
           "sample": "%d Stormer-Verlet steps of the N=%d liquid (FP64 linked cells, %d OpenMP threads)" %
                     (nsteps, n, cores)}
    if single:
        # one thread, on a 2-step sample of the first 131,072 particles of
        # the same lattice in a box of the same density (fcc 32^3 x 4)
        from paper_2505_03438_gb300 import scenarios
        small = scenarios.fcc_liquid(32, density=0.8442, temperature=0.72, seed=2)
        ps = oracle.make_params(small["box"], small["eps"], small["sigma"], small["rcut"], True)
        t0 = time.perf_counter()
        oracle.verlet_run(small["x"], small["v"], None, small["mass"], ps, small["dt"], 2, cell_min=cell_min, nthreads=1)
        t1 = time.perf_counter()
        m = len(small["x"])
        out["single_thread"] = {"value": m * 2 / (t1 - t0), "cores": 1, "seconds": t1 - t0,
                                "sample": "2 Stormer-Verlet steps of the same liquid at N=%d (fcc 32^3 x 4), one thread" % m}
    return out


def adjoint_leg(reps=20, nsteps=50, every=10):
    """Gradient workload (differentiable binary mixture, N = 32,768, FP32 pair
    math): wall time per call through the C ABI with device buffers, each
    call synchronising -- forces, force VJP, a 50-step checkpointed rollout
    and its reverse pass."""
    import numpy as np
    import torch

    import paper_2505_03438_gb300 as lj
    from paper_2505_03438_gb300 import scenarios

    sc = scenarios.binary_mixture()
    s = lj.System(sc, precision=0, stream=torch.cuda.current_stream().cuda_stream)
    n = s.n
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    cot = torch.randn((n, 3), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(7))
    g = torch.empty_like(F)

    def per_call(fn, k):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            fn()
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t0) / k

    out = {"workload": "binary_32768: KA-type 80:20 mixture, rho 1.2, rc 2.5 sigma_ab, FP32 pair math",
           "force_call_ms": per_call(lambda: lj.ljsel_compute(s.h, F), reps),
           "vjp_call_ms": per_call(lambda: lj.ljsel_force_vjp(s.h, cot, g, s.ntypes), reps)}
    xb = torch.randn((n, 3), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(8))
    gx, gv = torch.empty_like(xb), torch.empty_like(xb)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lj.ljsel_rollout(s.h, nsteps, every)
    t1 = time.perf_counter()
    lj.ljsel_rollout_vjp(s.h, xb, None, gx, gv, s.ntypes)
    t2 = time.perf_counter()
    out.update({"rollout_steps": nsteps, "checkpoint_every": every, "rollout_ms": 1e3 * (t1 - t0),
                "rollout_vjp_ms": 1e3 * (t2 - t1), "pairs_within_cutoff": s.pairs()[1]})
    s.close()
    return out


def batch_leg(peaks, steps=500, warmup=5, trial_steps=10, profile_steps=30, eager=False):
    """Batched replicas (512 periodic systems, N log-uniform in [256, 8192],
    about 1.17M particles): tile chosen by the batch autotuner, then `steps`
    steps in one graph launch timed with CUDA events on the batch's stream."""
    import torch

    import paper_2505_03438_gb300 as lj
    from paper_2505_03438_gb300 import scenarios

    reps = scenarios.replica_batch()
    stream = torch.cuda.current_stream()
    b = lj.Batch(reps, stream=stream.cuda_stream, use_graphs=not eager)
    t0 = time.perf_counter()
    chosen, costs = b.autotune(trial_steps=trial_steps)
    tune_s = time.perf_counter() - t0
    b.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0 = b.counters()
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    c1 = b.counters()
    prof = b.profile(profile_steps)
    npairs = len(b.pairs())
    fp32_peak = max(peaks["fp32_tflops"], peaks["fp32x2_tflops"])
    ach = npairs * FLOPS_PER_PAIR / (prof["force_ms"] * 1e-3) / 1e12 if prof["force_ms"] > 0 else None
    out = {"workload": "replicas_512: N log-uniform [256, 8192] (sum %d), rho U[0.3, 0.9], T U[0.7, 2.0], "
                       "rc 2.5, skin 0.3, R 10" % b.ntot,
           "value": b.ntot * steps / (ms * 1e-3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
           "graph_launches": 1, "tile": chosen.as_tuple(), "tile_costs_ms": costs, "tuning_s": tune_s,
           "rebuilds": c1["rebuilds"] - c0["rebuilds"], "early_rebuilds": c1["early_rebuilds"] - c0["early_rebuilds"],
           "steps_counted": c1["steps"] - c0["steps"], "capacity_retries": c1["capacity_retries"],
           "replica_rebuilds": c1["replica_rebuilds"] - c0["replica_rebuilds"],
           "pairs_within_cutoff": npairs,
           "kernel_ms": {k: prof[k] for k in ("rebuild_ms", "force_ms", "control_ms")},
           "roofline": {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": ach / fp32_peak if ach else None, "traffic": None,
                        "kernel": "batched force + update", "flops_per_launch": npairs * FLOPS_PER_PAIR,
                        "peak_basis": "measured FP32 probe (ljsel_measure_peaks)"}}
    b.close()
    return out


def inhomogeneous_leg(steps=20000, every=1000, strategies=("predictive", "expert"), fixed_steps=None,
                      skip_within=0.05, repeats=3):
    """Heated liquid ball (radius 40, density 0.8, T 3.0) in vapour (density
    0.01, T 1.2), periodic box 200, about 292k particles: `steps` steps with
    a tuning phase every `every` steps (trial steps count as steps; a phase
    whose live statistics moved less than skip_within since the last phase
    with trials is skipped), once with each of `strategies` and `repeats`
    times with the Random Forest strategy (the shipped forest; once more
    trialling its three most probable classes each phase), against the
    fixed configurations run over the same steps from the same state: every
    candidate screened over the first 1000 steps, the best five over all
    steps, the best two of those again so that each has `repeats` runs; the
    forest's runs and the fixed re-runs alternate, and the comparison is
    between medians."""
    import torch

    import paper_2505_03438_gb300 as lj
    from paper_2505_03438_gb300 import scenarios

    sc = scenarios.heated_sphere()
    n = len(sc["x"])
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def tuned_run(strat, top=1):
        phases = []
        s = lj.System(sc, stream=stream.cuda_stream)
        s.step(3)
        if strat == "forest":
            s.set_forest()

        def run():
            for k in range(steps // every):
                c, rep = s.autotune(strategy=strat, trial_steps=5, probe_steps=2, probe_factor=2.0,
                                    skip_within=skip_within, forest_top=top)
                s.step(every - rep["trial_steps_total"])
                phases.append({"step": k * every, "chosen": c.name(), "ntrialled": rep["ntrialled"],
                               "skipped": rep["skipped"], "phase_ms": rep["phase_ms"],
                               "overhead_ms": rep["overhead_ms"]})

        ms = timed(run)
        s.close()
        return {"value": n * steps / (ms * 1e-3), "strategy": strat,
                "phases_skipped": sum(p["skipped"] for p in phases),
                "tuning_overhead_ms": sum(p["overhead_ms"] for p in phases),
                "tuning_phase_ms": sum(p["phase_ms"] for p in phases), "phases": phases}

    probe = lj.System(sc)
    cands = lj.ljsel_default_candidates(probe.h)
    probe.close()

    def run_fixed(c, k):
        f = lj.System(sc, stream=stream.cuda_stream)
        try:
            lj.ljsel_set_config(f.h, c)
            f.step(3)
            return n * k / (timed(lambda: f.step(k)) * 1e-3)
        except lj.LjselError:
            return None
        finally:
            f.close()

    others = {st: tuned_run(st) for st in strategies}
    # the forest's three most probable classes trialled in each phase
    others["forest_top3"] = tuned_run("forest", 3)
    forest_runs = [tuned_run("forest")]
    screen = min(steps, 1000 if fixed_steps is None else fixed_steps)
    screened = {c.name(): (c, run_fixed(c, screen)) for c in cands}
    screened = {k: v for k, v in screened.items() if v[1] is not None}
    top = sorted(screened.values(), key=lambda cv: -cv[1])[:5]
    fixed = {c.name(): [run_fixed(c, steps)] for c, _ in top}
    fixed = {k: v for k, v in fixed.items() if v[0] is not None}
    byname = {c.name(): c for c, _ in top}
    best2 = sorted(fixed, key=lambda k: -fixed[k][0])[:2]
    for _ in range(repeats - 1):
        forest_runs.append(tuned_run("forest"))
        for k in best2:
            fixed[k].append(run_fixed(byname[k], steps))
    med = {k: statistics.median(v) for k, v in fixed.items() if len(v) == repeats}
    best = max(med.items(), key=lambda kv: kv[1]) if med else None
    forest_med = statistics.median(r["value"] for r in forest_runs)
    fr = dict(forest_runs[0], forest_top=1, values=[r["value"] for r in forest_runs], median=forest_med)
    out = {"workload": "heated_sphere: N=%d, box 200, ball r 40 rho 0.8 T 3.0, vapour rho 0.01 T 1.2, rc 2.5, "
                       "skin 0.3" % n,
           "unit": UNIT, "steps": steps, "retune_every": every, "skip_within": skip_within, "repeats": repeats,
           "forest": fr, "fixed_screen_steps": screen, "fixed_screened": {k: v[1] for k, v in screened.items()},
           "fixed": fixed, "best_fixed": best,
           "tuned_over_best_fixed": {"forest": forest_med / best[1] if best else None}}
    for st, r in others.items():
        out[st] = r
        out["tuned_over_best_fixed"][st] = r["value"] / best[1] if best else None
    return out


def walled_leg(steps=150000, every=1000, thermo_every=100, d_t=0.1, target=100.0,
               strategies=(("forest", "forest", 1), ("forest_top3", "forest", 3), ("predictive", "predictive", 1),
                           ("expert", "expert", 1)), repeats=3):
    """The walled heating sphere of Sec. 6 (5497 particles in a 200^3 box with
    reflective walls, cutoff 3, skin 0.5, R 10, dt 1e-4): every thermo_every
    steps a velocity-scaling thermostat moves T by at most d_t towards
    target; every `every` steps a tuning phase re-selects the configuration
    (its trial steps count as steps).  Each strategy's run and every fixed
    configuration run the same schedule from the same state; times are CUDA
    events on the system's stream around the whole run.  The Random Forest
    run (its first choice each phase) and the two best fixed configurations
    run `repeats` times, alternating, and compare by medians."""
    import torch

    import paper_2505_03438_gb300 as lj
    from paper_2505_03438_gb300 import scenarios

    sc = scenarios.walled_heating_sphere()
    n = len(sc["x"])
    stream = torch.cuda.current_stream()

    def schedule(s, strategy=None, phases=None, top=1):
        done, next_tune = 0, 0
        while done < steps:
            if strategy and done >= next_tune:
                c, rep = s.autotune(strategy=strategy, trial_steps=5, probe_steps=2, probe_factor=2.0, forest_top=top)
                done += rep["trial_steps_total"]
                phases.append((done, c.name(), rep["ntrialled"]))
                next_tune += every
            k = min(thermo_every - done % thermo_every, steps - done)
            s.step(k)
            done += k
            if done % thermo_every == 0:
                s.thermostat(target, d_t)
        return done

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), r

    out = {"workload": "walled_heating_sphere: N=%d, box 200 with reflective walls, rc 3, skin 0.5, R 10, dt 1e-4, "
                       "thermostat every %d steps by <= %g towards T %g, re-tune every %d" %
                       (n, thermo_every, d_t, target, every), "steps": steps}
    def tuned(label, strat, top):
        s = lj.System(sc, stream=stream.cuda_stream)
        if strat == "forest":
            s.set_forest()
        phases = []
        ms, done = timed(lambda: schedule(s, strat, phases, top))
        t_end = s.thermostat(target, 0.0)
        # the phases where the choice changed
        changes = [p for k, p in enumerate(phases) if k == 0 or p[1] != phases[k - 1][1]]
        s.close()
        return {"value": n * done / (ms * 1e-3), "steps": done, "final_T": t_end,
                "trials": sum(p[2] for p in phases), "choice_changes": changes[:40]}

    def run_fixed(c):
        f = lj.System(sc, stream=stream.cuda_stream)
        try:
            lj.ljsel_set_config(f.h, c)
            ms, done = timed(lambda: schedule(f))
            return n * done / (ms * 1e-3)
        except lj.LjselError:
            return None
        finally:
            f.close()

    for label, strat, top in strategies:
        out[label] = tuned(label, strat, top)
    probe = lj.System(sc)
    cands = {c.name(): c for c in lj.ljsel_default_candidates(probe.h)}
    probe.close()
    fixed = {k: v for k, v in ((name, run_fixed(c)) for name, c in cands.items()) if v is not None}
    runs = {k: [fixed[k]] for k in sorted(fixed, key=lambda k: -fixed[k])[:2]}
    forest_runs = [out["forest"]["value"]] if "forest" in out else []
    for _ in range(repeats - 1):
        if forest_runs:
            forest_runs.append(tuned("forest", "forest", 1)["value"])
        for k in runs:
            runs[k].append(run_fixed(cands[k]))
    med = {k: statistics.median(v) for k, v in runs.items()}
    best = max(med.items(), key=lambda kv: kv[1]) if med else None
    ratios = {label: out[label]["value"] / best[1] for label, _, _ in strategies} if best else None
    if best and forest_runs:
        out["forest"]["values"] = forest_runs
        ratios["forest"] = statistics.median(forest_runs) / best[1]
    out.update({"fixed": fixed, "fixed_reruns": runs, "best_fixed": best, "tuned_over_best_fixed": ratios})
    return out


def run_reference(args):
    """Reference arm: the oracle as it stands, on the host cores.  Every
    --steps step is a bounded sample (the budget scales with the requested
    steps); the line reports the steps actually timed."""
    from paper_2505_03438_gb300 import scenarios
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc = scenarios.liquid_1m()
    cb = oracle_rate(sc, budget_s=min(60.0, 6.0 + 2.0 * args.steps / 100.0))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": cb["steps"], "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * cb["seconds"] / cb["steps"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_2505_03438_gb300 as lj
    from paper_2505_03438_gb300 import forest as lj_forest
    from paper_2505_03438_gb300 import scenarios

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    sc = scenarios.liquid_1m()
    n = len(sc["x"])
    K, W = args.steps, args.warmup
    stream = torch.cuda.current_stream()
    x = torch.tensor(sc["x"], device="cuda")
    v = torch.tensor(sc["v"], device="cuda")
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    params = lj.make_params(sc["box"], skin=sc["skin"], dt=sc["dt"], use_graphs=not args.eager)
    peaks = lj.ljsel_measure_peaks(30.0)  # FP32, FP32x2, FP64 and reciprocal rates of this GPU
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    model = lj_forest.load()
    fixed_cfg = (lj.make_config(args.method, cluster_size=args.cluster, newton3=args.newton3,
                                threads_per_unit=args.tpu, rebuild_interval=sc["rebuild"], csf=args.csf)
                 if args.method else None)

    def barrier():
        if dist is not None:
            dist.barrier()

    def fresh():
        hh = lj.ljsel_create(params, n, x, v, t, stream.cuda_stream)
        if fixed_cfg is not None:
            lj.ljsel_set_config(hh, fixed_cfg)
        lj.ljsel_step(hh, W)  # warm-up
        torch.cuda.synchronize()
        return hh

    def timed(hh, strategy):
        """Timed region: one tuning phase (its trial steps count) + the rest of
        the K steps, bracketed by a barrier and device synchronisation.  The
        Random Forest strategy's forest is installed before it."""
        if strategy == "forest":
            lj.ljsel_set_forest(hh, model)
        c0 = lj.ljsel_get_counters(hh)
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = None
        if strategy:
            chosen, rep = lj.ljsel_autotune(hh, strategy=strategy, trial_steps=args.trial_steps,
                                            probe_steps=args.probe_steps, probe_factor=2.0)
            done = rep["trial_steps_total"]
        else:
            chosen, done = lj.ljsel_get_config(hh), 0
        lj.ljsel_step(hh, max(0, K - done))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        c1 = lj.ljsel_get_counters(hh)
        return {"ms": ms, "steps": c1["steps"] - c0["steps"], "chosen": chosen, "rep": rep,
                "rebuilds": c1["rebuilds"] - c0["rebuilds"], "early": c1["early_rebuilds"] - c0["early_rebuilds"]}

    headline = args.strategy if args.tune else None
    other = [st for st in ("expert", "full", "predictive", "forest") if args.tune and args.other and st != headline]
    extra_runs = {}
    for st in other:
        hx = fresh()
        r = timed(hx, st)
        extra_runs[st] = {"value": job_throughput(world, n, r["steps"], r["ms"]), "chosen": r["chosen"].name(),
                          "tuner": r["rep"]}
        lj.ljsel_destroy(hx)
    clk = Clocks(local)
    h = fresh()
    run = timed(h, headline)
    clocks = clk.stop()
    ms, steps_done, chosen, rep = run["ms"], run["steps"], run["chosen"], run["rep"]
    value = job_throughput(world, n, steps_done, ms)
    chosen_name = chosen.name()
    tuned_values = [value]

    def tuned_again():
        hx = fresh()
        r = timed(hx, headline)
        tuned_values.append(job_throughput(world, n, r["steps"], r["ms"]))
        lj.ljsel_destroy(hx)

    # ---- per-kernel timing (CUDA events around each launch) ---------------
    prof = lj.ljsel_profile_steps(h, args.profile_steps)
    _, npairs = lj.ljsel_get_pairs(h, 0)
    cnt = lj.ljsel_get_counters(h)

    # ---- every fixed configuration from the same initial state and the same
    # warm-up, then K timed steps that, like the tuned run's, include the
    # build of the configuration's neighbour structure (the state is set again
    # after the warm-up, which asks for a rebuild); the best three again,
    # alternating with further tuned runs, so that a drift of the GPU's speed
    # over the run weighs on both sides alike
    fixed, fixed_eff, best = {}, {}, None
    if args.fixed_steps != 0:
        kf = K if args.fixed_steps < 0 else args.fixed_steps
        cands = {c.name(): c for c in lj.ljsel_default_candidates(h)}

        def run_fixed(c):
            lj.ljsel_set_state(h, x, v)
            lj.ljsel_set_config(h, c)
            lj.ljsel_step(h, W)
            lj.ljsel_set_state(h, x, v)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lj.ljsel_step(h, kf)
            b.record(stream)
            torch.cuda.synchronize()
            return n * kf / (a.elapsed_time(b) * 1e-3)

        for name, c in cands.items():
            try:
                fixed[name] = run_fixed(c)
            except lj.LjselError:
                continue  # not available for this system
            ct = lj.ljsel_get_counters(h)
            _, np_c = lj.ljsel_get_pairs(h, 0)
            slots = ct["list_entries"] * (c.cluster_size if c.method == lj.METHOD_CLUSTER else 1)
            fixed_eff[name] = (np_c * (1 if c.newton3 else 2) / slots) if slots else None
        top = sorted(fixed, key=lambda k: -fixed[k])[:3]
        runs = {k: [] for k in top}
        for rr in range(max(1, args.repeats)):
            if rr > 0 and headline is not None:
                tuned_again()
            for k in top:
                runs[k].append(run_fixed(cands[k]))
        remeasured = {k: statistics.median(vv) for k, vv in runs.items()}
        bname = max(remeasured, key=remeasured.get)
        best = {"name": bname, "value": remeasured[bname], "steps": kf, "remeasured_top3": remeasured}
    else:
        for _ in range(max(0, args.repeats - 1)):
            if headline is not None:
                tuned_again()
    lj.ljsel_destroy(h)

    # ---- end to end through the C ABI with pinned host buffers ------------
    e2e = None
    if args.e2e:
        xp = torch.from_numpy(np.ascontiguousarray(sc["x"])).pin_memory()
        vp = torch.from_numpy(np.ascontiguousarray(sc["v"])).pin_memory()
        tp = torch.zeros(n, dtype=torch.int32).pin_memory()
        xo = torch.empty_like(xp).pin_memory()
        vo = torch.empty_like(vp).pin_memory()
        xh, vh, th, xoh, voh = xp.numpy(), vp.numpy(), tp.numpy(), xo.numpy(), vo.numpy()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        hp = lj.make_params(sc["box"], skin=sc["skin"], dt=sc["dt"], use_graphs=not args.eager)
        h2 = lj.ljsel_create(hp, n, xh, vh, th, stream.cuda_stream)
        done2 = 0
        if args.tune:
            if args.strategy == "forest":
                lj.ljsel_set_forest(h2, model)
            _, r2 = lj.ljsel_autotune(h2, strategy=args.strategy, trial_steps=args.trial_steps,
                                      probe_steps=args.probe_steps, probe_factor=2.0)
            done2 = r2["trial_steps_total"]
        lj.ljsel_step(h2, max(0, K - done2))
        lj.ljsel_get_state(h2, xoh, voh)
        t1 = time.perf_counter()
        lj.ljsel_destroy(h2)
        barrier()
        e2e = {"value": world * n * K / (t1 - t0), "unit": UNIT, "host_buffers": "pinned",
               "h2d_bytes_per_step": (xh.nbytes + vh.nbytes + th.nbytes) / K,
               "d2h_bytes_per_step": (xoh.nbytes + voh.nbytes) / K}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    emit(args, locals())
    if dist is not None:
        dist.destroy_process_group()


def emit(args, L):
    """Rank 0: the compact headline line (printed last) and the details file."""
    import paper_2505_03438_gb300 as lj
    sc, n, K, W, prof, peaks, chosen, rep, run = (L[k] for k in ("sc", "n", "K", "W", "prof", "peaks", "chosen",
                                                                  "rep", "run"))
    npairs, cnt, hbm, world = L["npairs"], L["cnt"], L["hbm"], L["world"]
    ms, steps_done, value = L["ms"], L["steps_done"], L["value"]
    chosen_name = chosen.name()
    # ---- roofline of the dominant kernel (force, fused with the update when
    # N3L is off), against the measured FP32 peak of this GPU -----------------
    fp32_peak = max(peaks["fp32_tflops"], peaks["fp32x2_tflops"])
    force_ms = prof["force_ms"]
    achieved = npairs * FLOPS_PER_PAIR / (force_ms * 1e-3) / 1e12 if force_ms > 0 else None
    base = "-".join(chosen_name.split("-")[:3])
    traffic = FORCE_TRAFFIC_1M.get(base) if (chosen.csf == 1.0 and n == 1048576) else None
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": (achieved / fp32_peak) if achieved else None, "traffic": traffic,
            "traffic_source": ("ncu capture of %s at N = 1,048,576" % base) if traffic else None,
            "kernel": "force (%s)" % chosen_name, "launch_ms": force_ms,
            "flops_per_launch": npairs * FLOPS_PER_PAIR, "peak_basis": "of measured (FP32 probe)"}
    # ---- step roofline -------------------------------------------------------
    rl = 2.5 + sc["skin"]
    entries_alg = npairs * (rl / 2.5) ** 3  # unordered pairs within the list radius
    nc1 = int((sc["box"][0] / (rl * (1 + 1.0 / 4096) ** 2)))
    rebuild_every = steps_done / max(run["rebuilds"], 1)
    sr = step_roofline(n, npairs, True, entries_alg, nc1 ** 3, rebuild_every, peaks, hbm)
    ms_step = ms / max(steps_done, 1)
    sr["t_measured_us"] = 1e3 * ms_step
    sr["frac"] = sr["t_roof_us"] / sr["t_measured_us"]
    best = L["best"]
    tuned_med = statistics.median(L["tuned_values"])
    comparison = None
    if best:
        comparison = {"tuned_median": tuned_med, "best_fixed": best["name"], "best_fixed_median": best["value"],
                      "ratio": tuned_med / best["value"], "repeats": args.repeats, "steps": K}
    cb = None
    if args.cpu_baseline and world == 1:
        cb = oracle_rate(sc, single=True)
    details = {"peaks_probe": peaks, "hbm_gbs": hbm, "fixed": L["fixed"], "fixed_pair_efficiency": L["fixed_eff"],
               "best_fixed": best, "tuned_values": L["tuned_values"], "other_tuned_runs": L["extra_runs"],
               "tuner": dict(rep, strategy=L["headline"]) if rep else None,
               "kernel_ms": {k: prof[k] for k in ("rebuild_ms", "force_ms", "update_ms", "control_ms")},
               "counters": cnt, "pairs_within_cutoff": npairs, "rebuilds": run["rebuilds"],
               "early_rebuilds": run["early"], "step_roofline": sr}
    if args.adjoint:
        details["adjoint"] = adjoint_leg()
    if args.batch:
        details["batch"] = batch_leg(peaks)
    if args.inhomo:
        details["inhomogeneous"] = inhomogeneous_leg(fixed_steps=args.inhomo_fixed_steps)
    if args.walled:
        details["walled_heating_sphere"] = walled_leg(steps=args.walled_steps)
    # kernels launched in the timed region.  Graph steps: the force (and the
    # update when N3L is on) and the control kernel, the rebuild chain when a
    # rebuild runs, and the loop-init and command kernels of each call.
    # Tuning trials run as plain launches: every trial step launches the
    # whole chain (its kernels return at once unless a rebuild is due), and
    # each trial first builds its structure.  A phase also launches its three
    # statistics kernels.
    n3 = 1 if chosen.newton3 else 0
    chain = 5 + {lj.METHOD_VL: 1, lj.METHOD_CLUSTER: 2, lj.METHOD_VLW: 2}.get(chosen.method, 0)
    trial_steps = rep["trial_steps_total"] if rep else 0
    ntrial = rep["ntrialled"] if rep else 0
    graph_steps = steps_done - trial_steps
    graph_rebuilds = max(0, run["rebuilds"] - ntrial)
    launches = int(trial_steps * (chain + 2 + n3) + ntrial * (chain + 3) + graph_steps * (2 + n3) +
                   graph_rebuilds * chain + 4 + (3 if rep else 0))
    path = args.details
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(details, f, indent=1, default=str)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": int(steps_done),
        "warmup": W, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (state + lists > 129 MB)", "tuned": bool(args.tune),
                   "strategy": L["headline"], "chosen": chosen_name,
                   "precision": "FP32 pair math, FP64 integration and sums"},
        "roofline": roof,
        "step_roofline": {"t_roof_us": sr["t_roof_us"], "t_measured_us": sr["t_measured_us"], "frac": sr["frac"]},
        "tuned_vs_best_fixed": comparison,
        "cpu_baseline": cb,
        "e2e": L["e2e"],
        "clocks": L["clocks"],
        "gpu_launches": launches,
        "details": os.path.relpath(path, ROOT),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--method", default=None, help="run this fixed method (LC, VL, VLW, CL) from the start")
    ap.add_argument("--newton3", action="store_true")
    ap.add_argument("--tpu", type=int, default=1)
    ap.add_argument("--cluster", type=int, default=4)
    ap.add_argument("--csf", type=float, default=1.0, help="with --method: cell size factor (1.0 or 0.5)")
    ap.add_argument("--trial-steps", type=int, default=5)
    ap.add_argument("--probe-steps", type=int, default=2)
    ap.add_argument("--strategy", default="forest", choices=["full", "predictive", "expert", "forest"],
                    help="tuning strategy of the headline run (the others are reported in the details)")
    ap.add_argument("--repeats", type=int, default=3,
                    help="tuned runs and re-runs of the three best fixed configurations for the medians")
    ap.add_argument("--fixed-steps", type=int, default=-1, help="steps per fixed configuration (-1: same as --steps)")
    ap.add_argument("--profile-steps", type=int, default=60)
    ap.add_argument("--details", default=os.path.join(ROOT, "_build", "bench_details.json"))
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--eager", action="store_true", help="plain stream launches instead of the step graph")
    ap.add_argument("--no-other", dest="other", action="store_false", help="skip the other tuning strategies")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false", help="skip the gradient-workload timings")
    ap.add_argument("--no-batch", dest="batch", action="store_false", help="skip the batched-replica run")
    ap.add_argument("--no-inhomo", dest="inhomo", action="store_false", help="skip the heated-sphere re-tuning run")
    ap.add_argument("--inhomo-fixed-steps", type=int, default=None,
                    help="screening steps per fixed configuration in the heated-sphere comparison (default 1000; "
                         "the best five then run all 20000 steps)")
    ap.add_argument("--no-walled", dest="walled", action="store_false", help="skip the walled heating-sphere run")
    ap.add_argument("--walled-steps", type=int, default=60000,
                    help="steps of the walled heating-sphere run (the paper heats for 150000)")
    ap.add_argument("--leg", default="all", choices=["all", "batch", "adjoint", "inhomo", "walled"],
                    help="run only one leg and print its JSON")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.leg == "batch":
        import paper_2505_03438_gb300 as lj
        print(json.dumps(batch_leg(lj.ljsel_measure_peaks(30.0), steps=args.steps, warmup=args.warmup,
                                   eager=args.eager)), flush=True)
    elif args.leg == "adjoint":
        print(json.dumps(adjoint_leg()), flush=True)
    elif args.leg == "inhomo":
        print(json.dumps(inhomogeneous_leg(fixed_steps=args.inhomo_fixed_steps)), flush=True)
    elif args.leg == "walled":
        print(json.dumps(walled_leg(steps=args.walled_steps)), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
