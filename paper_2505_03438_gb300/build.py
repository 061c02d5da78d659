"""Build the CUDA library libljsel.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically.  The result lives in
``paper_2505_03438_gb300/_build/`` (git-ignored).  The checked variant
libljsel_checked.so is compiled with -DLJSEL_CHECK: the kernels check list,
cell and slot indices against their arrays and report a failure instead of
touching memory outside them (select it with LJSEL_LIBRARY=checked).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libljsel.so")
SOURCES = ["rebuild.cu", "force.cu", "cluster.cu", "window.cu", "system.cu", "capi.cu", "noalloc.cu", "adjoint.cu", "batch.cu", "probe.cu"]
HEADERS = ["ljsel_internal.cuh", "kernels.cuh", "system.h", "update.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libljsel")


def _flags():
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-O3", "-diag-suppress", "128",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _jobs(variant, force, extra):
    """(compile commands, objects, library path) of one variant."""
    out = OUT if variant == "plain" else os.path.join(OUT, variant)
    lib = LIB if variant == "plain" else os.path.join(OUT, "libljsel_%s.so" % variant)
    flags = _flags() + (["-DLJSEL_CHECK"] if variant == "checked" else [])
    os.makedirs(out, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "ljsel.h")]
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s, *hdrs]):
            jobs.append([nvcc(), *flags, *extra, "-c", s, "-o", o])
    return jobs, objs, lib


def _run(cmd, verbose=False):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose and (r.stdout or r.stderr):
        sys.stderr.write(r.stdout + r.stderr)


def build(force: bool = False, verbose: bool = False, extra=(), variants=("plain", "checked")) -> str:
    """Compile the library variants (all translation units in one thread
    pool) and link them; returns the path of the plain library."""
    os.makedirs(OUT, exist_ok=True)
    plans = [(v, *_jobs(v, force, extra)) for v in variants]
    jobs = [j for _, js, _, _ in plans for j in js]
    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(lambda c: _run(c, verbose), jobs))
    for _, js, objs, lib in plans:
        if force or js or _stale(lib, objs):
            tmp = lib + ".tmp.%d" % os.getpid()
            _run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"])
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
