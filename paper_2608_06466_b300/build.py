"""Build libmc.so (the C-ABI burn library) in-tree with nvcc for sm_103a.

Each csrc/*.cu file is compiled to its own object in parallel, then linked
into paper_2608_06466_b300/libmc.so. Objects are rebuilt when their source or
any header is newer. `build(check=True)` (or `--check`) builds the same
sources with -DMC_BOUNDS_CHECK into libmc_check.so, the bounds-check build
(include/mc.h, mc_bounds_report)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys
import time

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(ROOT, "_build", "obj")
LIB = os.path.join(PKG, "libmc.so")
OBJ_CHECK = os.path.join(ROOT, "_build", "obj_check")
LIB_CHECK = os.path.join(PKG, "libmc_check.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-I" + INCLUDE, "-I" + CSRC]


def _newest(paths):
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def build(force: bool = False, verbose: bool = False, extra_flags=None, check: bool = False) -> str:
    obj_dir = OBJ_CHECK if check else OBJ
    lib = LIB_CHECK if check else LIB
    if check:
        extra_flags = list(extra_flags or []) + ["-DMC_BOUNDS_CHECK"]
    os.makedirs(obj_dir, exist_ok=True)
    # objects carry the time the build started, so that a source or header
    # edited while it runs is newer than every object compiled from the old
    # text and the next build compiles them again
    t_start = time.time()
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    t_hdr = _newest(headers)
    flags = FLAGS + list(extra_flags or [])
    jobs = []
    for src in sources:
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), t_hdr):
            jobs.append((src, obj))

    def compile_one(job):
        src, obj = job
        cmd = [NVCC] + ARCH + flags + ["-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        os.utime(obj, (t_start, t_start))
        return src, r.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
            for src, err in ex.map(compile_one, jobs):
                if verbose and err.strip():
                    print(f"[{os.path.basename(src)}]\n{err}", file=sys.stderr)
    objs = [os.path.join(obj_dir, os.path.basename(s)[:-3] + ".o") for s in sources]
    if force or jobs or not os.path.exists(lib) or os.path.getmtime(lib) < _newest(objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
        os.utime(lib, (t_start, t_start))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, check="--check" in sys.argv))
