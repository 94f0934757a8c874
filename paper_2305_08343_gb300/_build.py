"""In-tree build of the native libraries (no cmake, no setuptools).

* ``libscenegen.so``  — the seeded input generators alone (gcc).
* ``libsubcull.so``   — the product: host builders (g++), CUDA kernels for
  sm_103a (nvcc), the seeded generators, and the C-ABI of include/subcull.h.

Translation units compile in parallel; a unit is rebuilt only when a source
or header it may include is newer than its object.
"""
from __future__ import annotations

import glob
import os
import platform
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
# per-architecture output: objects built on one host type never mix with another's
OUT = os.path.join(PKG, "_build", platform.machine() or "unknown")
INCLUDE = os.path.join(ROOT, "include")

ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsubcull")


def _cuda_home() -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(_nvcc())))


def _newest(paths) -> float:
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build_scenegen(force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libscenegen.so")
    srcs = [os.path.join(CSRC, "gen", "scenegen.c"), os.path.join(CSRC, "gen", "scenegen.h")]
    if not force and os.path.exists(so) and os.path.getmtime(so) >= _newest(srcs):
        return so
    tmp = so + f".tmp{os.getpid()}"
    _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
          "-fno-fast-math", srcs[0], "-o", tmp, "-lm"])
    os.replace(tmp, so)
    return so


HOST_FLAGS = ["-O2", "-fPIC", "-std=c++17", "-pthread", "-ffp-contract=off",
              "-fno-fast-math", "-Wall", "-Wno-unused-function"]
# Test ops (slab, Alg. 1 quantisation, Moeller-Trumbore) must be plain IEEE
# float operations: no FMA contraction, IEEE division/sqrt, denormals kept.
NVCC_FLAGS = [ARCH, "-lineinfo", "-O3", "-std=c++17", "-fmad=false", "-prec-div=true",
              "-prec-sqrt=true", "-ftz=false", "-Xcompiler", "-fPIC",
              "-Xptxas", "-warn-spills", "--expt-relaxed-constexpr"]


def product_sources():
    return (sorted(glob.glob(os.path.join(CSRC, "host", "*.cpp")))
            + sorted(glob.glob(os.path.join(CSRC, "cuda", "*.cu")))
            + [os.path.join(CSRC, "gen", "scenegen.c")])


def _headers():
    return (glob.glob(os.path.join(CSRC, "**", "*.h"), recursive=True)
            + glob.glob(os.path.join(CSRC, "**", "*.cuh"), recursive=True)
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def build_product(force: bool = False, verbose: bool = False) -> str:
    """Compiles and links libsubcull.so; returns its path."""
    os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
    so = os.path.join(OUT, "libsubcull.so")
    hdr_time = _newest(_headers())
    srcs = product_sources()
    nvcc = _nvcc()
    incs = ["-I" + INCLUDE, "-I" + CSRC, "-I" + os.path.join(_cuda_home(), "include")]
    jobs = []
    objs = []
    for s in srcs:
        base = os.path.relpath(s, CSRC).replace(os.sep, "_")
        obj = os.path.join(OUT, "obj", base + ".o")
        objs.append(obj)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(
                os.path.getmtime(s), hdr_time, os.path.getmtime(__file__)):
            continue
        if s.endswith(".cu"):
            cmd = [nvcc, *NVCC_FLAGS, *incs, "-c", s, "-o", obj]
        elif s.endswith(".c"):
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
                   *incs, "-c", s, "-o", obj]
        else:
            cmd = ["g++", *HOST_FLAGS, *incs, "-c", s, "-o", obj]
        jobs.append(cmd)
    logs = []
    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            logs = list(ex.map(_run, jobs))
    if force or jobs or not os.path.exists(so) or os.path.getmtime(so) < _newest(objs):
        tmp = so + f".tmp{os.getpid()}"
        _run([nvcc, ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"])
        os.replace(tmp, so)
    if verbose:
        for lg in logs:
            if lg.strip():
                print(lg)
    return so


def build_all(force: bool = False, verbose: bool = False):
    return build_scenegen(force), build_product(force, verbose)
