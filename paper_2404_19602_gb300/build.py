"""Build the CUDA library libpgc.so for sm_103a (GB300) in-tree.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_2404_19602_gb300/_build/libpgc.so`` against the shared CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpgc.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpgc.so")


ONE_D = "pgc_inst_1d.cu"   # compiled once per one-dimensional shape


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu") and f != ONE_D)


def shapes_1d():
    """Basis sizes P of the one-dimensional shapes (the PGC_SHAPES_1D list of pgc_runner.h)."""
    src = open(os.path.join(CSRC, "pgc_runner.h")).read()
    m = re.search(r"#define PGC_SHAPES_1D\(X\)(.*)", src)
    return [int(v) for v in re.findall(r"X\((\d+)\)", m.group(1))]


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "pgc.h")]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    deps = _deps()
    if not force and not _stale(LIB, deps):
        return LIB
    flags = FLAGS + list(extra_flags or [])
    objs = []
    cmds = []
    for P in sorted(shapes_1d(), reverse=True):   # the largest units first
        obj = os.path.join(BUILD, "pgc_inst_1d_%d.o" % P)
        objs.append(obj)
        cmds.append([nvcc] + ARCH + flags + ["-DPGC_1D_P=%d" % P, "-c", os.path.join(CSRC, ONE_D), "-o", obj])
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmds.append([nvcc] + ARCH + flags + ["-c", src, "-o", obj])
    cmds.sort(key=lambda c: "21x36" not in c[-3])   # the longest unit first (stable otherwise)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 1, len(cmds)))) as ex:
        for out in ex.map(run, cmds):
            if verbose and out:
                print(out, file=sys.stderr)
    tmp = LIB + ".tmp%d" % os.getpid()
    run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-lpthread", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
