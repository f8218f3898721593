"""Builds libset.so in-tree: nvcc for the sm_103a stage kernels, g++ for the host runtime.

Objects go to ``_build/`` and the library to ``lib/`` beside this file (both git-ignored).
Translation units compile in parallel; one ``-gencode`` (compute_103a -> sm_103a).  No CMake.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libset.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["kernels/blur_hist.cu", "kernels/saxpy_scan_max.cu", "kernels/img_sobel_hist.cu",
              "kernels/mlp_ln.cu", "kernels/hotspot.cu", "kernels/guards.cu", "kernels/plan.cu",
              "kernels/dev_dispatch.cu", "kernels/copy.cu"]
CPP_SOURCES = ["runtime/executor.cpp", "runtime/layout.cpp", "runtime/cuda_device.cpp", "runtime/capi.cpp",
               "runtime/trace.cpp", "runtime/dev_dispatch.cpp", "runtime/dd_cuda.cpp"]
HEADERS = ["kernels/stages.h", "kernels/params.h", "kernels/tc.cuh", "kernels/cp_async.cuh", "kernels/dev_dispatch.h",
           "runtime/executor.h", "runtime/sync.h", "runtime/layout.h", "runtime/thread_error.h", "runtime/dd_backend.h"]

INCLUDES = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", os.path.join(CUDA_HOME, "include")]
NVCC_FLAGS = GENCODE + ["-O3", "-lineinfo", "-std=c++20", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                        "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
CXX_FLAGS = ["-O2", "-std=c++20", "-fPIC", "-Wall", "-Wno-unused-function", "-ffp-contract=off"]


def _obj(src: str) -> str:
    return os.path.join(BUILD, src.replace("/", "_") + ".o")


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, extra_nvcc=()) -> str:
    """Compiles every source that changed and links lib/libset.so; returns its path."""
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "set.h"), __file__]
    jobs = []
    for src in CU_SOURCES:
        s, o = os.path.join(CSRC, src), _obj(src)
        if force or _stale(o, [s] + headers):
            jobs.append([NVCC] + NVCC_FLAGS + list(extra_nvcc) + INCLUDES + ["-c", s, "-o", o])
    for src in CPP_SOURCES:
        s, o = os.path.join(CSRC, src), _obj(src)
        if force or _stale(o, [s] + headers):
            jobs.append(["g++"] + CXX_FLAGS + INCLUDES + ["-c", s, "-o", o])
    with ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as pool:
        for out in pool.map(_run, jobs):
            if verbose and out.strip():
                sys.stdout.write(out)
    objs = [_obj(s) for s in CU_SOURCES + CPP_SOURCES]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([NVCC] + GENCODE + ["-shared", "-cudart", "shared", "-o", tmp] + objs +
             ["-Xlinker", "-rpath=" + os.path.join(CUDA_HOME, "lib64"), "-lpthread", "-ldl"])
        os.replace(tmp, LIB)
    return LIB


def ptxas_report() -> str:
    """Registers / spills / shared memory of every kernel (-Xptxas -v), for review."""
    out = []
    for src in CU_SOURCES:
        out.append(_run([NVCC] + NVCC_FLAGS + ["-Xptxas", "-v"] + INCLUDES +
                        ["-c", os.path.join(CSRC, src), "-o", os.devnull]))
    return "\n".join(out)


def clean() -> None:
    shutil.rmtree(BUILD, ignore_errors=True)
    if os.path.exists(LIB):
        os.remove(LIB)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
    if "--ptxas" in sys.argv:
        print(ptxas_report())
