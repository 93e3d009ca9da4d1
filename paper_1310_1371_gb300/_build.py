"""Build the detector's shared library (librd.so) in-tree for sm_103a.

Each CUDA translation unit is compiled by its own nvcc process (in parallel),
then linked into ``paper_1310_1371_gb300/_lib/librd.so`` with the CUDA
runtime linked statically.  Host code is compiled with -ffp-contract=off: the
weight tables must be computed with one rounding per operation.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "librd.so")
SOURCES = ["rd_api.cu", "k_stencil.cu", "k_vote.cu", "k_fit.cu", "k_soft.cu", "rd_serve.cu", "rd_static.cu",
           "rd_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
                     "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


VARIANTS = {
    None: (OBJ, LIB, []),
    # debug build: data-dependent indices checked in the kernels (RD_OVF_CHECK)
    "check": (os.path.join(PKG, "_build_check"), os.path.join(LIBDIR, "librd_check.so"), ["-DRD_CHECK"]),
}


def lib_path(variant: str | None = None) -> str:
    return LIB if variant is None else VARIANTS[variant][1]


def build(verbose: bool = False, extra: list[str] | None = None, force: bool = False,
          variant: str | None = None) -> str:
    """Compile (only what changed) and return the path of librd.so (or of a
    named variant: "check", the bounds-checked debug build librd_check.so)."""
    obj_dir, lib, vflags = (OBJ, LIB, []) if variant is None else VARIANTS[variant]
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "rd.h"))
    flags = NVCC_FLAGS + vflags + (extra or [])
    procs, objs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(obj_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [nvcc(), "-c", s, "-o", o] + flags
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    if force or procs or _stale(lib, objs):
        cmd = [nvcc(), "-shared", "-o", lib] + objs + ARCH + ["-Xcompiler", "-fPIC", "-lpthread"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
