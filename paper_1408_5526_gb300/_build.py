"""Build librqmc.so (the CUDA C-ABI library) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel to an object file under
``_build/`` and then linked into ``paper_1408_5526_gb300/librqmc.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "librqmc.so")
SOURCES = ["api.cu", "setup.cu", "probe.cu", "k_points.cu", "k_product.cu", "k_lmm.cu", "k_lmm_halton.cu", "k_lmm_sobol.cu",
           "k_lmm_philox.cu", "k_lmm_loaded.cu", "k_mbs.cu", "noalloc.cu", "k_adjoint.cu", "k_adjoint_halton.cu",
           "k_adjoint_sobol.cu", "k_adjoint_philox.cu", "k_adjoint_loaded.cu", "batch.cu", "k_batch.cu", "k_batch_halton.cu",
           "k_batch_sobol.cu", "k_batch_philox.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librqmc.so")


def flags(extra=()):
    return ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "-Xcompiler", "-Wno-unknown-pragmas",
                   "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                   "-diag-suppress", "177"] + list(extra)


def _stale(obj, src) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(ROOT, "include", "rqmc.h"))
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(o, s):
            jobs.append([cc, "-c", s, "-o", o] + flags(extra))
    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        run([cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared", "-Xlinker",
                                                      "-rpath,/usr/local/cuda/lib64"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
