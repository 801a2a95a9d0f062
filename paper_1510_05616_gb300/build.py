"""Build libstokes.so (and the bounds-checked libstokes_debug.so) in-tree with nvcc for sm_103a,
one translation unit per .cu, in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libstokes.so")
# the same sources with the device bounds checks compiled in (-DSTOKES_DEBUG)
LIB_DEBUG = os.path.join(HERE, "libstokes_debug.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libstokes")
    return p


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    files = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return max(os.path.getmtime(f) for f in files)


def up_to_date() -> bool:
    dep = _deps()
    return all(os.path.exists(p) and os.path.getmtime(p) >= dep for p in (LIB, LIB_DEBUG))


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every csrc/*.cu twice -- the release library libstokes.so and the debug library
    libstokes_debug.so (device bounds checks) -- in parallel, and link both; returns the
    release library's path."""
    if not force and up_to_date():
        return LIB
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    variants = {LIB: (os.path.join(BUILD, "release"), []),
                LIB_DEBUG: (os.path.join(BUILD, "debug"), ["-DSTOKES_DEBUG"])}
    jobs = []
    for lib, (odir, defs) in variants.items():
        os.makedirs(odir, exist_ok=True)
        jobs += [(src, odir, defs) for src in sources()]

    def compile_one(job):
        src, odir, defs = job
        obj = os.path.join(odir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *defs, *extra, "-I", INCLUDE, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose or ptxas_info:
        for _, log in results:
            if log.strip():
                print(log)
    for lib, (odir, _) in variants.items():
        objs = [o for o, _ in results if os.path.dirname(o) == odir]
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [cc, *ARCH, "-shared", "-o", tmp] + objs + [
            "-lcublas", "-lcusolver", "-Xlinker", "-rpath=" + os.path.join(os.path.dirname(os.path.dirname(cc)), "lib64")]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
