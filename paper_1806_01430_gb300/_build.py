"""Build libgao.so in-tree: nvcc for the CUDA sources (sm_103a only), g++ for the
host runtime, linked with the static CUDA runtime.  Sources compile in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgao.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["kernels_ew.cu", "gemm_simt.cu", "gemm_tc.cu", "residual.cu"]
CPP = ["runtime.cpp", "cpu_loops.cpp", "ga_engine.cpp", "batch.cpp"]


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")] + [
        os.path.join(HERE, "..", "include", "gao.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, extra_nvcc=()) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    inc = ["-I", CSRC, "-I", os.path.join(HERE, "..", "include")]
    jobs = []
    for f in CU:
        o = os.path.join(OUT, f + ".o")
        jobs.append(([NVCC, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
                      "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", *inc, *extra_nvcc,
                      "-c", os.path.join(CSRC, f), "-o", o], o))
    for f in CPP:
        o = os.path.join(OUT, f + ".o")
        jobs.append((["g++", "-std=c++17", "-O3", "-fPIC", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                      "-Wall", "-Wno-unused-function", *inc, "-I", os.path.join(CUDA_HOME, "include"),
                      "-c", os.path.join(CSRC, f), "-o", o], o))
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        logs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for l in logs:
            if l.strip():
                print(l, file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    _run([NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *[o for _, o in jobs],
          "-Xcompiler", "-fopenmp", "-lgomp", "-lpthread", "-ldl", "-lrt"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
