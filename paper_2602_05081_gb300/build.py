"""Build libgf.so (the CUDA C-ABI library) in-tree for sm_103a with nvcc.

Translation units compile in parallel; the result lands at
``paper_2602_05081_gb300/_build/libgf.so``.  Rebuilds only when a source or
header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgf")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + [os.path.join(ROOT, "include", "gf.h")]


def flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                   "-I" + os.path.join(ROOT, "include"), "--expt-relaxed-constexpr",
                   "-Xptxas", "-O3"]


def build(force: bool = False, verbose: bool = False, variant: str | None = None,
          defines=()) -> str:
    """Compile libgf.so.  `variant` builds a separately named library with extra
    preprocessor `defines` (e.g. variant="timers", defines=["GF_PHASE_TIMERS"])."""
    if variant:
        return _build_into(os.path.join(HERE, "_build_" + variant), force, verbose, defines)
    return _build_into(BUILD, force, verbose, ())


def _build_into(build_dir, force, verbose, defines):
    lib = os.path.join(build_dir, "libgf.so")
    os.makedirs(build_dir, exist_ok=True)
    if not force and os.path.exists(lib):
        newest = max(os.path.getmtime(p) for p in _deps())
        if os.path.getmtime(lib) >= newest:
            return lib
    nvcc = _nvcc()
    objs = []
    cmds = []
    for src in _sources():
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        cmds.append([nvcc, *flags(), *("-D" + d for d in defines), "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return r

    with cf.ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
        list(ex.map(run, cmds))
    tmp = lib + ".tmp%d" % os.getpid()
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    if "--timers" in sys.argv:
        print(build(force="--force" in sys.argv, verbose=True, variant="timers",
                    defines=["GF_PHASE_TIMERS"]))
    else:
        print(build(force="--force" in sys.argv, verbose=True))
