"""Build libsph.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into one shared
library next to this file.  No PyTorch headers are involved: the library has a
plain C ABI (include/sph.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsph.so")

SOURCES = ["sph_sort.cu", "sph_build.cu", "sph_pairs.cu", "sph_pairs_m6.cu", "sph_pairs_m4_wrap.cu",
           "sph_pairs_m6_wrap.cu", "sph_gravity.cu", "sph_block.cu", "sph_integrate.cu", "sph_export.cu", "sph_api.cu", "sph_server.cu",
           "sph_noalloc.cu", "sph_peak.cu"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-O2", "-Xptxas", "-O3", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsph.so")


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(CSRC, "sph_internal.cuh"), os.path.join(CSRC, "sph_tuned.h"),
            os.path.join(CSRC, "sph_pairs.cuh"), os.path.join(CSRC, "sph_leaf.cuh"), os.path.join(ROOT, "include", "sph.h")]
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose: bool = False, force: bool = False, extra: list | None = None,
          out: str | None = None, build_dir: str | None = None) -> str:
    """Compile the sources (in parallel) and link libsph.so.  `extra` adds
    nvcc flags (e.g. -D overrides of launch-shape constants); `out` and
    `build_dir` redirect the outputs."""
    lib = out or LIB
    bdir = build_dir or BUILD
    os.makedirs(bdir, exist_ok=True)
    exe = nvcc()
    flags = NVFLAGS + (extra or [])
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(bdir, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, src):
            jobs.append([exe, *ARCH, *flags, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return r

    with cf.ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        list(ex.map(run, jobs))
    if jobs or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        run([exe, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(verbose=True, force="--force" in sys.argv))
