"""Build liblamino.so (the CUDA path) in-tree for sm_103a.

    python -m paper_2511_01893_b300.build [--verbose] [--checked]

Compiles every ``csrc/*.cu`` with nvcc for ``arch=compute_103a,code=sm_103a``
and links them into ``paper_2511_01893_b300/liblamino.so``.  Objects go to
``_build/`` at the repository root.  Rebuilds only what changed.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "liblamino.so")
# the same sources with LAM_BOUNDS_CHECK defined: index checks that record a
# failing site in the plan's error word instead of accessing out of range
LIB_CHECKED = os.path.join(HERE, "liblamino_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _deps_mtime(src: str) -> float:
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers += [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    return max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in headers])


def build(verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Build liblamino.so, or with checked=True liblamino_checked.so (the
    LAM_BOUNDS_CHECK variant, objects under _build/checked)."""
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    lib = LIB_CHECKED if checked else LIB
    if checked:
        extra_flags = ("-DLAM_BOUNDS_CHECK", *extra_flags)
    os.makedirs(bdir, exist_ok=True)
    objs, jobs = [], []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith(".cu"):
            continue
        src = os.path.join(CSRC, f)
        obj = os.path.join(bdir, f[:-3] + ".o")
        objs.append(obj)
        if os.path.exists(obj) and os.path.getmtime(obj) >= _deps_mtime(src) and list(extra_flags) in (
                [], ["-DLAM_BOUNDS_CHECK"]):
            continue
        jobs.append([NVCC, *FLAGS, *extra_flags, "-c", src, "-o", obj])
    # the translation units compile independently: run them side by side
    # (capturing each one's output so that messages do not interleave)
    procs = []
    for cmd in jobs:
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    failed = None
    for cmd, p in zip(jobs, procs):
        out, _ = p.communicate()
        if out:
            sys.stdout.write(out)
            sys.stdout.flush()
        if p.returncode != 0 and failed is None:
            failed = subprocess.CalledProcessError(p.returncode, cmd)
    if failed is not None:
        raise failed
    if (not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs)
            or jobs):
        cmd = [NVCC, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", lib, *objs, "-lcudart", "-ldl"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
    return lib


if __name__ == "__main__":
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(verbose="--verbose" in sys.argv, extra_flags=extra, checked="--checked" in sys.argv))
