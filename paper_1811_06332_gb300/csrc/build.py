"""Builds libfmm_gb300.so in-tree for sm_103a.

Runs the table/kernel generator, compiles every translation unit with nvcc
in parallel (one -gencode, compute_103a -> sm_103a), and links a shared
library next to the Python binding.  Object files go to csrc/_build/.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
ROOT = os.path.dirname(PKG)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(PKG, "libfmm_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include"), "-I" + HERE, "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    sys.path.insert(0, HERE)
    import gen  # noqa: E402  (generator lives beside this file)
    gen.generate()
    hand = sorted(glob.glob(os.path.join(HERE, "*.cu")))
    generated = sorted(glob.glob(os.path.join(HERE, "_gen", "*.cu")))
    return hand + generated


def _compile(src: str, extra) -> str:
    rel = os.path.relpath(src, HERE).replace(os.sep, "_")
    obj = os.path.join(BUILD, rel + ".o")
    deps = [src] + glob.glob(os.path.join(HERE, "*.h")) + glob.glob(os.path.join(HERE, "*.cuh")) + \
        glob.glob(os.path.join(HERE, "_gen", "*.h")) + [os.path.join(ROOT, "include", "fmm_gb300.h")]
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    cmd = [nvcc()] + ARCH + FLAGS + list(extra) + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr[-6000:]))
    if r.stderr.strip() and os.environ.get("FMM_BUILD_VERBOSE"):
        print(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(jobs: int | None = None, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    jobs = jobs or max(1, min(len(srcs), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr[-4000:]))
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(extra=sys.argv[1:]))
