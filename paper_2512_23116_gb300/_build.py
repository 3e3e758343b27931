"""Build of the in-tree CUDA library liblbm_gb300.so (sm_103a only).

Each translation unit under csrc/ is compiled by nvcc in parallel with
``-gencode arch=compute_103a,code=sm_103a``; the objects are linked into one
shared library with the static CUDA runtime and cuFFT.  Only the ``lbm_*``
symbols of include/lbm.h are exported.

The same sources are also built with ``-DLBM_BOUNDS_CHECK`` into
liblbm_gb300_checked.so: every device index is checked and a failed check is
reported as an error instead of being performed (the stand-in for a device
memory checker; the binding loads it when LBM_LIBRARY=checked).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "liblbm_gb300.so")
LIB_CHECKED = os.path.join(HERE, "liblbm_gb300_checked.so")
BUILD_DIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -ftz=true: FP32 subnormals flush to zero, so the MUFU reciprocals and square
# roots of the collision need no subnormal fix-up code.  Populations, moments and
# velocities are far above the FP32 subnormal range; the one quantity that can
# fall into it, |S|^2 of a nearly relaxed cell, is taken as zero below 1e-30
# in any case.
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-ftz=true", "-Xcompiler", "-fPIC,-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode())
                h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Build liblbm_gb300.so and liblbm_gb300_checked.so (when their sources
    changed); returns the path of the first."""
    variants = [(LIB, []), (LIB_CHECKED, ["-DLBM_BOUNDS_CHECK"])]
    dig = _digest()
    todo = []
    for lib, defs in variants:
        stamp = lib + ".stamp"
        if not force and os.path.exists(lib) and os.path.exists(stamp):
            with open(stamp) as fh:
                if fh.read().strip() == dig:
                    continue
        todo.append((lib, defs))
    if not todo:
        return LIB
    nvcc = _nvcc()
    srcs = _sources()

    def compile_one(job):
        src, tag, defs = job
        out_dir = os.path.join(BUILD_DIR, tag)
        os.makedirs(out_dir, exist_ok=True)
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    jobs = [(src, os.path.basename(lib).replace(".so", ""), defs) for lib, defs in todo for src in srcs]
    with cf.ThreadPoolExecutor(max_workers=min(max(1, os.cpu_count() or 1), len(jobs), 16)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for k, (lib, _) in enumerate(todo):
        mine = objs[k * len(srcs):(k + 1) * len(srcs)]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *mine, "-cudart", "static", "-lcufft",
               "-Xlinker", "--exclude-libs,ALL"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
        with open(lib + ".stamp", "w") as fh:
            fh.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
