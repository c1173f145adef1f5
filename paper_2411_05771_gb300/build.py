"""Builds libskei.so in-tree for sm_103a with nvcc (no torch extension
machinery: the library exposes a plain C ABI)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libskei.so")
# the bounds-check build (SKEI_CHECK = 1), objects of its own
CHECK_DIR = os.path.join(PKG, "_build_check")
CHECK_LIB = os.path.join(CHECK_DIR, "libskei_check.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libskei")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(extra_flags, lib=LIB, out_dir=OUT_DIR) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    deps += [os.path.join(INCLUDE, "skei.h"), os.path.abspath(__file__)]
    stamp = os.path.join(out_dir, "flags.txt")
    flags = " ".join(ARCH + NVCC_FLAGS + list(extra_flags))
    if not os.path.exists(stamp) or open(stamp).read() != flags:
        return True
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), check: bool = False) -> str:
    """Compile every csrc/*.cu for sm_103a and link libskei.so (check: the
    bounds-check build libskei_check.so, SKEI_CHECK = 1).  Returns its path."""
    lib, out_dir = (CHECK_LIB, CHECK_DIR) if check else (LIB, OUT_DIR)
    extra_flags = list(extra_flags) + (["-DSKEI_CHECK=1"] if check else [])
    if not force and not _stale(extra_flags, lib, out_dir):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stderr}")
    os.replace(tmp, lib)
    with open(os.path.join(out_dir, "flags.txt"), "w") as f:
        f.write(" ".join(ARCH + NVCC_FLAGS + list(extra_flags)))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
