"""Builds the in-tree CUDA library libpxc.so for sm_103a (B300) with nvcc."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))
DEPS = SRC + sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh"))) + [os.path.join(ROOT, "include", "pxc.h")]
LIB = os.path.join(HERE, "libpxc.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def flags(extra=()):
    return ARCH + list(extra) + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
                   "-Xptxas", "-v", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                   "-I", os.path.join(HERE, "csrc")]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose: bool = False, out: str | None = None, defines=()) -> str:
    """Compile csrc/*.cu into libpxc.so (or `out`, with extra -D `defines` for tuning builds)."""
    lib = out or LIB
    if out is None and not force and not stale():
        return LIB
    objdir = os.path.join(HERE, "_build") if out is None else \
        os.path.join(os.path.dirname(os.path.abspath(out)), "_build_" + os.path.basename(out).replace(".", "_"))
    os.makedirs(objdir, exist_ok=True)
    objs = []
    for src in SRC:
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [NVCC, "-c", src, "-o", obj] + flags([f"-D{d}" for d in defines])
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError(f"nvcc failed on {src}")
        if verbose:
            sys.stderr.write(r.stderr)
        with open(obj + ".ptxas.txt", "w") as f:
            f.write(r.stderr)
        objs.append(obj)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
