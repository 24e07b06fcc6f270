"""Compile the CUDA library libsdcef.so for sm_103a (in-tree, no cmake).

The solver kernel is instantiated once per (threads per column, Krylov
precision) pair in its own translation unit; the units compile in parallel
and are linked with the host-side C ABI into one shared library.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsdcef.so")
# the bounds-checking build (-DSDCEF_CHECKS; see csrc/checks.cuh)
BUILD_CHECKS = os.path.join(HERE, "_build_checks")
LIB_CHECKS = os.path.join(BUILD_CHECKS, "libsdcef.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]
# (threads per column, Krylov type, preconditioner type) of each kernel instance
INSTANCES = [(tpb, kr, pr) for kr, pr in (("double", "double"), ("float", "float"),
                                          ("double", "sdcef::dfloat"))
             for tpb in (32, 64, 128, 256)]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsdcef.so")


def _sources():
    out = []
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def _digest(flags) -> str:
    h = hashlib.sha256()
    for p in _sources():
        h.update(p.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + flags).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    """Build (or reuse) libsdcef.so; returns its path. checks=True builds the
    bounds-checking variant into _build_checks/ instead."""
    build_dir, lib = (BUILD_CHECKS, LIB_CHECKS) if checks else (BUILD, LIB)
    flags = FLAGS + (["-DSDCEF_CHECKS"] if checks else [])
    os.makedirs(build_dir, exist_ok=True)
    stamp = os.path.join(build_dir, "libsdcef.stamp")
    dig = _digest(flags)
    if not force and os.path.exists(lib) and os.path.exists(stamp) and open(stamp).read() == dig:
        return lib
    nvcc = _nvcc()
    jobs = []
    for tpb, kr, pr in INSTANCES:
        obj = os.path.join(build_dir, f"kern_{tpb}_{kr}_{pr.split(':')[-1]}.o")
        cmd = [nvcc, *ARCH, *flags, f"-DSDCEF_TPB={tpb}", f"-DSDCEF_KR={kr}", f"-DSDCEF_PR={pr}"]
        if (tpb, kr, pr) == INSTANCES[0]:
            cmd.append("-DSDCEF_WITH_ORDER")
        cmd += ["-c", os.path.join(CSRC, "kern_inst.cu"), "-o", obj]
        jobs.append((obj, cmd))
    for var in ("MG", "TAB"):
        obj = os.path.join(build_dir, f"kern_{var.lower()}.o")
        jobs.append((obj, [nvcc, *ARCH, *flags, f"-DSDCEF_{var}", "-c",
                           os.path.join(CSRC, "kern_inst.cu"), "-o", obj]))
    for src in ("sdcef.cu", "noalloc.cu", "mlp.cu", "fields.cu", "probe.cu"):
        obj = os.path.join(build_dir, src.replace(".cu", "_host.o"))
        jobs.append((obj, [nvcc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]))

    def run(job):
        obj, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {obj}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(run, jobs))
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(dig)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checks="--checks" in sys.argv))
