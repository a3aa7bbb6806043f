"""Build libdpd.so in-tree with nvcc for sm_103a, and the portable CPU
library libdpd_cpu.so with the host C compiler.

Each translation unit under ``csrc/`` is compiled to an object file in
``_build/`` (in parallel, skipped when up to date), then linked into
``lib/libdpd.so``.  The CUDA runtime is linked statically, so the library only
needs the driver at run time.  ``cpu/dpd_cpu.c`` becomes ``lib/libdpd_cpu.so``
(C11, OpenMP, GCC vector extensions; no architecture flags, so the same source
builds on x86-64 and AArch64).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ_DIR = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "lib")
LIB_PATH = os.path.join(LIB_DIR, "libdpd.so")
CPU_SRC = os.path.join(HERE, "cpu", "dpd_cpu.c")
CPU_LIB_PATH = os.path.join(LIB_DIR, "libdpd_cpu.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code: fused multiply-adds allowed (the FP64 condition estimate's matrix
# products are its largest host cost).
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=fast", "-I", INCLUDE,
              "--expt-relaxed-constexpr", "-Xcompiler", "-Wall"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdpd")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, verbose_ptxas=False):
    obj = os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o")
    if not _stale(obj, [src, *_headers()]):
        return obj, ""
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj + ".tmp"]
    if verbose_ptxas:
        cmd[1:1] = ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj, r.stderr


def build_cpu(force: bool = False) -> str:
    """lib/libdpd_cpu.so from cpu/dpd_cpu.c with the host C compiler."""
    os.makedirs(LIB_DIR, exist_ok=True)
    deps = [CPU_SRC, os.path.join(INCLUDE, "dpd_cpu.h")]
    if force or _stale(CPU_LIB_PATH, deps):
        cc = os.environ.get("CC", "gcc")
        tmp = CPU_LIB_PATH + f".tmp{os.getpid()}"
        cmd = [cc, "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=fast", "-Wall",
               "-o", tmp, CPU_SRC]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"{cc} failed for {CPU_SRC}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, CPU_LIB_PATH)
    return CPU_LIB_PATH


def build(jobs: int | None = None, verbose_ptxas: bool = False, force: bool = False) -> str:
    os.makedirs(OBJ_DIR, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    srcs = _sources()
    if force:
        for s in srcs:
            o = os.path.join(OBJ_DIR, os.path.basename(s)[:-3] + ".o")
            if os.path.exists(o):
                os.remove(o)
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas), srcs))
    objs = [o for o, _ in results]
    if verbose_ptxas:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    if _stale(LIB_PATH, objs):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(verbose_ptxas=v, force="--force" in sys.argv), file=sys.stderr)
    print(build_cpu(force="--force" in sys.argv), file=sys.stderr)
