"""Builds the host-simulation test library (executor + simulated device, no CUDA) and its
sanitizer stress drivers.  Test infrastructure only."""
from __future__ import annotations

import ctypes
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RT = os.path.join(ROOT, "paper_2606_05495_gb300", "csrc", "runtime")
SIM = os.path.join(ROOT, "tests", "hostsim")
OUT = os.path.join(SIM, "_build")
SOURCES = ([os.path.join(RT, f) for f in ("executor.cpp", "layout.cpp", "capi.cpp", "dev_dispatch.cpp")] +
           [os.path.join(SIM, f) for f in ("sim_device.cpp", "sim_dd.cpp")])
FLAGS = ["-std=c++20", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", RT, "-I",
         os.path.join(ROOT, "paper_2606_05495_gb300", "csrc"), "-pthread"]


def _newer(target, deps):
    return os.path.exists(target) and all(os.path.getmtime(target) >= os.path.getmtime(d) for d in deps)


def _deps():
    hdrs = ([os.path.join(RT, h) for h in ("executor.h", "sync.h", "layout.h", "dd_backend.h")] +
            [os.path.join(ROOT, "include", "set.h"),
             os.path.join(ROOT, "paper_2606_05495_gb300", "csrc", "kernels", "dev_dispatch.h")])
    return SOURCES + hdrs


def build_lib() -> str:
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libset_hostsim.so")
    if not _newer(so, _deps()):
        subprocess.check_call(["g++", "-O2", "-shared", "-o", so + ".tmp"] + FLAGS + SOURCES)
        os.replace(so + ".tmp", so)
    return so


def build_stress(sanitizer: str, driver: str = "stress") -> str:
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, f"{driver}_{sanitizer}")
    src = os.path.join(SIM, driver + ".cpp")
    if not _newer(exe, _deps() + [src]):
        subprocess.check_call(["g++", "-O1", "-g", f"-fsanitize={sanitizer}", "-o", exe + ".tmp"] + FLAGS +
                              SOURCES + [src])
        os.replace(exe + ".tmp", exe)
    return exe


def load(env=None):
    """Loads a fresh copy of the simulation library (environment read at set_create time)."""
    if env:
        os.environ.update({k: str(v) for k, v in env.items()})
    return ctypes.CDLL(build_lib())
