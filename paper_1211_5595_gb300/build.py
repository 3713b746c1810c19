"""Builds librc.so (the C-ABI CUDA library, csrc/*.cu) and librc_probe.so
(the bandwidth probes of include/rc_probe.h, csrc/probe/*.cu) in-tree with nvcc
for sm_103a.

Each .cu file compiles to an object in parallel, then nvcc links each shared
library (static CUDA runtime). Host code is compiled without floating-point
contraction so the FP64 camera record rounds exactly as specified.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librc.so")
PROBE_DIR = os.path.join(CSRC, "probe")
PROBE_LIB = os.path.join(PKG, "librc_probe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources(d=CSRC):
    return sorted(os.path.join(d, f) for f in os.listdir(d) if f.endswith(".cu"))


def _deps_mtime(d, headers):
    files = sources(d) + [os.path.join(d, f) for f in os.listdir(d) if f.endswith((".h", ".cuh"))]
    files += [os.path.join(INCLUDE, h) for h in headers]
    return max(os.path.getmtime(f) for f in files)


def _build_lib(lib, src_dir, headers, tag, force, verbose, extra_flags):
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime(src_dir, headers):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, tag + os.path.basename(src)[:-3] + ".o")
        cmd = [nv, *ARCH, *FLAGS, *extra_flags, "-I", INCLUDE, "-I", src_dir, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources(src_dir)))
    tmp = lib + ".tmp"
    cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


DEBUG_LIB = os.path.join(PKG, "librc_debug.so")


def build_debug(force: bool = False, verbose: bool = False) -> str:
    """librc_debug.so: the same library compiled with -DRC_DEBUG (every brick
    and table index checked on the device, failures reported as a status)."""
    return _build_lib(DEBUG_LIB, CSRC, ["rc.h"], "debug_", force, verbose, ("-DRC_DEBUG",))


def build_probe(force: bool = False, verbose: bool = False) -> str:
    """librc_probe.so: the bandwidth probes the bench's rooflines use."""
    return _build_lib(PROBE_LIB, PROBE_DIR, ["rc_probe.h"], "probe_", force, verbose, ())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """librc.so, with librc_debug.so and librc_probe.so beside it; returns
    librc.so's path."""
    with cf.ThreadPoolExecutor(max_workers=3) as ex:
        probe = ex.submit(build_probe, force, verbose)
        debug = ex.submit(build_debug, force, verbose)
        lib = _build_lib(LIB, CSRC, ["rc.h"], "", force, verbose, extra_flags)
        probe.result()
        debug.result()
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []))
