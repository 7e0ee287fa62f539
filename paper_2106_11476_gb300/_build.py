"""Build libfw2.so in-tree with nvcc for sm_103a (no cmake, one -gencode).

Translation units compile in parallel into ``_build/`` and link into
``paper_2106_11476_gb300/libfw2.so``.  Set FW2_PTXAS_VERBOSE=1 to print the
register / shared-memory report of every kernel.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfw2.so")
SOURCES = ["api.cu", "prep.cu", "aux.cu", "step2d.cu", "step2d_pipe.cu", "step3d.cu", "step3d_pipe.cu", "noalloc.cu", "batch.cu",
           "fit.cpp"]
# second compilations of a source: (source, object name, extra flags); the
# tile kernels for 5..8 mechanisms build beside those for 0..4
VARIANTS = [("step2d.cu", "step2d_wide", ["-DFW2_WIDE_RELAX"]), ("step3d.cu", "step3d_wide", ["-DFW2_WIDE_RELAX"])]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _flags():
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if os.environ.get("FW2_PTXAS_VERBOSE"):
        f += ["-Xptxas", "-v"]
    return f


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "fw2.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(job):
        src, name, extra = job
        obj = os.path.join(BUILD, name + ".o")
        cmd = [nvcc] + _flags() + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or os.environ.get("FW2_PTXAS_VERBOSE"):
            sys.stderr.write(r.stderr)
        return obj

    jobs = [(src, os.path.splitext(src)[0], []) for src in SOURCES] + VARIANTS
    # the longest compilations first
    heavy = ("step3d.cu", "step3d_pipe.cu", "step2d.cu")
    jobs.sort(key=lambda j: j[0] not in heavy)
    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
