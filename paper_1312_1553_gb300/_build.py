"""Build of the nle CUDA library (libnle.so) for sm_103a.

The kernels are compiled once per (precision, rows-per-thread, triangular-
solve schedule) triple in parallel translation units, then linked with the C ABI and the host set-up
code into ``paper_1312_1553_gb300/libnle.so``.  Objects go to ``_build/`` at
the repository root.  A stamp over the sources and flags skips rebuilds.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libnle.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
           "--expt-relaxed-constexpr"] + ARCH
# (tag, precision, rows-per-thread chunks, chain schedule of the triangular solves)
VARIANTS = [(f"{p}{r}{'c' if c else ''}", t, r, c) for c in (0, 1) for p, t in (("f", "float"), ("d", "double"))
            for r in (1, 2, 4, 8)]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp", ".h", ".cuh"))) + [
        os.path.join(ROOT, "include", "nle.h")]


def _stamp() -> str:
    h = hashlib.sha256()
    for f in _sources():
        with open(f, "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    h.update(" ".join(NVFLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile libnle.so if the sources changed; return its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp_file = os.path.join(BUILD, "libnle.stamp")
    stamp = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as fh:
            if fh.read().strip() == stamp:
                return LIB
    nvcc = _nvcc()
    cmds = []
    objs = []
    kern = os.path.join(CSRC, "nle_kernels.cu")
    for tag, typ, rpc, chain in VARIANTS:
        o = os.path.join(BUILD, f"nle_kernels_{tag}.o")
        cmds.append([nvcc, *NVFLAGS, f"-DNLE_T={typ}", f"-DNLE_RPC={rpc}", f"-DNLE_TAG={tag}",
                     f"-DNLE_CHAIN_TU={chain}", "-c", kern, "-o", o])
        objs.append(o)
    for src in ("nle_api.cu", "nle_setup.cpp", "nle_noalloc.cu", "nle_ict.cu"):
        o = os.path.join(BUILD, src.replace(".", "_") + ".o")
        # the IC factor must round exactly like the host factor: no contraction
        extra = ["-fmad=false"] if src == "nle_ict.cu" else []
        cmds.append([nvcc, *NVFLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", o])
        objs.append(o)
    jobs = jobs or min(len(cmds), max(1, os.cpu_count() or 1))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            print(r.stdout + r.stderr)
        return r

    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        list(ex.map(run, cmds))
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
