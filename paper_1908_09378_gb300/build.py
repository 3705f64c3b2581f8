"""Build the CUDA library (libpbh.so) in-tree for sm_103a with nvcc.

One -gencode; the host ABI and each kernel are separate translation units
compiled in parallel, so the build takes about as long as its slowest kernel.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libpbh.so")
# the host ABI and one translation unit per kernel, compiled in parallel
SOURCES = [os.path.join(CSRC, f) for f in ("pbh.cu", "k_op.cu", "k_ops.cu", "k_grid.cu", "k_cluster.cu", "k_cta.cu",
                                           "k_batch.cu", "k_serve.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in ("core.cuh", "concurrent.cuh", "heapop.cuh", "plan.h", "kernels.h")] + \
    [os.path.join(INCLUDE, "pbh.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpbh.so")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in DEPS)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    objdir = tempfile.mkdtemp(prefix="obj", dir=LIBDIR)
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    if extra:
        flags[0:0] = extra
    try:
        procs = []
        for src in SOURCES:
            obj = os.path.join(objdir, os.path.basename(src) + ".o")
            procs.append((src, obj, subprocess.Popen([nvcc(), *flags, "-c", "-o", obj, src],
                                                     stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        failed = False
        for src, obj, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                failed = True
                sys.stderr.write(f"nvcc failed on {os.path.basename(src)}:\n{out}")
            elif verbose:
                sys.stderr.write(out)
        if failed:
            raise RuntimeError("nvcc failed building libpbh.so")
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=LIBDIR)
        os.close(fd)
        res = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *[o for _, o, _ in procs]],
                             capture_output=True, text=True)
        if res.returncode != 0:
            if os.path.exists(tmp):
                os.unlink(tmp)
            sys.stderr.write(res.stdout + res.stderr)
            raise RuntimeError("nvcc failed linking libpbh.so")
        os.replace(tmp, LIB)
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
