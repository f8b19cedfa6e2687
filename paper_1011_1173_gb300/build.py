"""Build the CUDA library (``libchm.so``) in-tree for sm_103a.

Each ``csrc/*.cu`` / ``csrc/*.cpp`` translation unit is compiled in parallel
with nvcc into ``_build/`` and linked into one shared library whose exported
symbols are the C ABI declared in ``include/chm.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libchm.so")
# the bounds-checked variant (-DCHM_CHECK): every global index of the kernels checked
OUT_CHECK = os.path.join(PKG, "_build_check")
LIB_CHECK = os.path.join(OUT_CHECK, "libchm_check.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--prec-div=true", "--prec-sqrt=true", "--fmad=true", "-I" + INCLUDE, "-I" + SRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(SRC, "*.cu")) + glob.glob(os.path.join(SRC, "*.cpp")))


def _headers():
    return (glob.glob(os.path.join(SRC, "*.cuh")) + glob.glob(os.path.join(SRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _plan(out_dir, lib, extra, force, verbose, srcs, hdrs, nvcc):
    """Compile jobs and objects of one variant of the library."""
    os.makedirs(out_dir, exist_ok=True)
    objs, jobs = [], []
    for s in srcs:
        o = os.path.join(out_dir, os.path.basename(s) + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc] + ARCH + NVCC_FLAGS + extra + ["-c", s, "-o", o + ".tmp"]
            if verbose:
                cmd.append("-Xptxas=-v")
            jobs.append((cmd, o))
    return objs, jobs


def _link(lib, objs, nvcc):
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "--cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stdout))
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Compile and link ``libchm.so`` and (``checked``) its bounds-checked
    variant ``libchm_check.so`` (the same sources with -DCHM_CHECK); the
    translation units of both compile in one parallel pool.  Returns the
    path of ``libchm.so``."""
    srcs = _sources()
    hdrs = _headers()
    nvcc = _nvcc()
    variants = [(OUT, LIB, [])] + ([(OUT_CHECK, LIB_CHECK, ["-DCHM_CHECK"])] if checked else [])
    plans = [(lib,) + _plan(out_dir, lib, extra, force, verbose, srcs, hdrs, nvcc)
             for out_dir, lib, extra in variants]
    jobs = [j for _, _, js in plans for j in js]

    def run(job):
        cmd, o = job
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stdout))
        os.replace(o + ".tmp", o)
        return r.stdout

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(max(8, os.cpu_count() or 8), len(jobs))) as ex:
            for out in ex.map(run, jobs):
                if verbose and out:
                    sys.stdout.write(out)
    for lib, objs, js in plans:
        if force or js or _stale(lib, objs):
            _link(lib, objs, nvcc)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
