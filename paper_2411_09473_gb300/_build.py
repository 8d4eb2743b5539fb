"""Build the CUDA library (libimm_gb300.so) in-tree with nvcc for sm_103a.

Each .cu file under csrc/ is compiled to an object in parallel, then the
objects are linked into a shared library with the CUDA runtime linked
statically.  Host code is compiled without FMA contraction so the fp64 theta
control rounds the same way as any plain IEEE evaluation.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB_NAME = "libimm_gb300.so"
LIB_PATH = os.path.join(OUT_DIR, LIB_NAME)
# The bounds-checked variant (-DIMM_BOUNDS_CHECK): every checked index is
# compared with its buffer's bound and the first violation is reported as an
# error instead of being used.  Tests load it in a process of its own.
BOUNDS_LIB_PATH = os.path.join(OUT_DIR, "libimm_gb300_bounds.so")
VARIANTS = {"": (LIB_PATH, "obj", []), "bounds": (BOUNDS_LIB_PATH, "obj_bounds", ["-DIMM_BOUNDS_CHECK"])}

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
              "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(path: str = LIB_PATH) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None, variant: str = "") -> str:
    lib_path, obj_name, vflags = VARIANTS[variant]
    if not force and not _stale(lib_path):
        return lib_path
    os.makedirs(OUT_DIR, exist_ok=True)
    obj_dir = os.path.join(OUT_DIR, obj_name)
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    flags = ARCH + NVCC_FLAGS + vflags + list(extra_flags or [])

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        cmd = [cc] + flags + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, flush=True)
        return obj

    srcs = sources()
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


def build_all(force: bool = False) -> None:
    """The library and its bounds-checked variant, compiled side by side."""
    with concurrent.futures.ThreadPoolExecutor(max_workers=2) as ex:
        list(ex.map(lambda v: build(force=force, variant=v), ["", "bounds"]))


if __name__ == "__main__":
    print(build(force=True, verbose=True))
