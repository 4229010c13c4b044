"""Build libpolymul.so and libpolymul_probe.so (sm_103a) in-tree with nvcc.

Each .cu file compiles to an object in parallel, then the shared libraries are
linked next to this file: libpolymul.so from csrc/*.cu (the product's C-ABI,
include/polymul.h) and libpolymul_probe.so from csrc/probe/*.cu (the
roofline's register-only probes, include/polymul_probe.h).  Usage:
``python -m paper_1303_7425_gb300.build``.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpolymul.so")
PROBE_LIB = os.path.join(HERE, "libpolymul_probe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources(sub=""):
    return sorted(glob.glob(os.path.join(CSRC, sub, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile both libraries (objects in parallel); returns libpolymul.so's path."""
    os.makedirs(BUILD, exist_ok=True)
    hdrs = _headers()
    targets = [(LIB, _sources()), (PROBE_LIB, _sources("probe"))]
    jobs = []
    objs_of = []
    for _, srcs in targets:
        objs = []
        for s in srcs:
            o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
            objs.append(o)
            if force or _stale(o, [s] + hdrs):
                jobs.append([nvcc()] + ARCH + NVCC_FLAGS + list(extra_flags) + ["-c", s, "-o", o])
        objs_of.append(objs)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
                if verbose or res.returncode:
                    sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
                if res.returncode:
                    raise RuntimeError(f"nvcc failed: {cmd[-3]}")
    for (lib, _), objs in zip(targets, objs_of):
        if force or jobs or _stale(lib, objs):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
            res = subprocess.run(cmd, capture_output=True, text=True)
            if res.returncode:
                sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
                raise RuntimeError("link failed")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
