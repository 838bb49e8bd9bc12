"""Build of the CUDA library ``_build/liblbm.so`` for sm_103a (nvcc, no cmake).

lbm_ops.cu is compiled once per (lattice, storage) pair and once more per 3D pair for z-slab
contexts, lbm_host.cu and lbm_noalloc.cu once; the twenty-seven objects build in parallel and
link against the shared CUDA runtime, which the process shares with PyTorch.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "liblbm.so")
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing"]
LATTICES = (9, 19, 27)
STORAGES = (0, 1, 2, 3, 4)
SLAB_LATTICES = (19, 27)


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(INCLUDE, "lbm.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile and link liblbm.so if any source is newer than it; returns its path."""
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OUT, exist_ok=True)
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    jobs = jobs or min(16, os.cpu_count() or 4)
    tasks = []
    for q in LATTICES:
        for s in STORAGES:
            obj = os.path.join(OUT, f"lbm_ops_q{q}_s{s}.o")
            tasks.append([nvcc, *ARCH, *FLAGS, f"-DLBM_Q={q}", f"-DLBM_S={s}", "-c",
                          os.path.join(CSRC, "lbm_ops.cu"), "-o", obj])
    for q in SLAB_LATTICES:  # the same kernels with the first processed plane at 1 (z-slabs)
        for s in STORAGES:
            obj = os.path.join(OUT, f"lbm_ops_q{q}_s{s}_slab.o")
            tasks.append([nvcc, *ARCH, *FLAGS, f"-DLBM_Q={q}", f"-DLBM_S={s}", "-DLBM_SLAB=1", "-c",
                          os.path.join(CSRC, "lbm_ops.cu"), "-o", obj])
    for name in ("lbm_host", "lbm_noalloc"):
        tasks.append([nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, name + ".cu"), "-o",
                      os.path.join(OUT, name + ".o")])
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        logs = list(ex.map(_run, tasks))
    if verbose:
        print("\n".join(logs))
    objs = [t[t.index("-o") + 1] for t in tasks]
    tmp = LIB + f".tmp{os.getpid()}"
    _run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
          "-Xlinker", "-rpath", "-Xlinker", cuda_lib])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=False))
