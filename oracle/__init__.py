"""CPU oracle of the SET executor's workloads (plain, serial, fp64 where the GPU reassociates).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package.  It shares no code with
the CUDA path (paper_2606_05495_gb300); both read inputs from ``datagen``.

``oracle.c`` holds the integer and fp32 stages (compiled to liboracle.so and
called through ctypes, which releases the GIL so jobs can run on many host
threads); ``mlp.py`` holds the fp64 MLP / LayerNorm job.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import mlp  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so beside this file (plain gcc, no FP contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            vp, i32, sz, f32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float, ctypes.c_double
            sig = {
                "oracle_blur3x3": ([vp, i32, i32, vp], None),
                "oracle_hist256": ([vp, sz, vp], None),
                "oracle_saxpy": ([f32, vp, vp, sz, vp], None),
                "oracle_exscan": ([vp, sz, vp, vp], None),
                "oracle_maxabs": ([vp, sz], f64),
                "oracle_gray": ([vp, i32, i32, vp], None),
                "oracle_gauss5": ([vp, i32, i32, vp], None),
                "oracle_sobel": ([vp, i32, i32, vp], None),
                "oracle_job_blur_hist": ([vp, i32, i32, vp, vp], None),
                "oracle_job_saxpy_scan_max": ([f32, vp, vp, sz, vp, vp, vp], f64),
                "oracle_job_img_sobel_hist": ([vp, i32, i32, vp, vp, vp, vp], None),
                "oracle_hotspot_params": ([i32, i32, vp], None),
                "oracle_hotspot": ([vp, vp, i32, i32, i32, vp], None),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes, fn.restype = args, res
            _lib = L
    return _lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def blur3x3(img: np.ndarray) -> np.ndarray:
    img = _c(img, np.uint8)
    H, W = img.shape
    out = np.empty_like(img)
    lib().oracle_blur3x3(img.ctypes.data, W, H, out.ctypes.data)
    return out


def hist256(img: np.ndarray) -> np.ndarray:
    img = _c(img, np.uint8)
    h = np.empty(256, np.uint32)
    lib().oracle_hist256(img.ctypes.data, img.size, h.ctypes.data)
    return h


def saxpy(a: float, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    x, y = _c(x, np.float32), _c(y, np.float32)
    z = np.empty_like(x)
    lib().oracle_saxpy(a, x.ctypes.data, y.ctypes.data, x.size, z.ctypes.data)
    return z


def exscan(z: np.ndarray):
    """(S, A): fp64 exclusive prefix sum of z and the running absolute sum."""
    z = _c(z, np.float32)
    S = np.empty(z.size, np.float64)
    A = np.empty(z.size, np.float64)
    lib().oracle_exscan(z.ctypes.data, z.size, S.ctypes.data, A.ctypes.data)
    return S, A


def maxabs(S: np.ndarray) -> float:
    S = _c(S, np.float64)
    return float(lib().oracle_maxabs(S.ctypes.data, S.size))


def gray(rgb: np.ndarray) -> np.ndarray:
    rgb = _c(rgb, np.uint8)
    H, W, _ = rgb.shape
    g = np.empty((H, W), np.uint8)
    lib().oracle_gray(rgb.ctypes.data, W, H, g.ctypes.data)
    return g


def gauss5(g: np.ndarray) -> np.ndarray:
    g = _c(g, np.uint8)
    H, W = g.shape
    q = np.empty_like(g)
    lib().oracle_gauss5(g.ctypes.data, W, H, q.ctypes.data)
    return q


def sobel(q: np.ndarray) -> np.ndarray:
    q = _c(q, np.uint8)
    H, W = q.shape
    s = np.empty_like(q)
    lib().oracle_sobel(q.ctypes.data, W, H, s.ctypes.data)
    return s


def job_blur_hist(img: np.ndarray):
    """(blurred image, histogram of the blurred image)."""
    img = _c(img, np.uint8)
    H, W = img.shape
    out = np.empty_like(img)
    h = np.empty(256, np.uint32)
    lib().oracle_job_blur_hist(img.ctypes.data, W, H, out.ctypes.data, h.ctypes.data)
    return out, h


def job_saxpy_scan_max(a: float, x: np.ndarray, y: np.ndarray):
    """(z fp32, S fp64, A fp64, m fp64) of one scan job."""
    x, y = _c(x, np.float32), _c(y, np.float32)
    n = x.size
    z = np.empty(n, np.float32)
    S = np.empty(n, np.float64)
    A = np.empty(n, np.float64)
    m = lib().oracle_job_saxpy_scan_max(a, x.ctypes.data, y.ctypes.data, n, z.ctypes.data,
                                        S.ctypes.data, A.ctypes.data)
    return z, S, A, float(m)


def job_img_sobel_hist(rgb: np.ndarray):
    """(Sobel image, histogram of the Sobel image) of one image job."""
    rgb = _c(rgb, np.uint8)
    H, W, _ = rgb.shape
    g = np.empty((H, W), np.uint8)
    q = np.empty((H, W), np.uint8)
    s = np.empty((H, W), np.uint8)
    h = np.empty(256, np.uint32)
    lib().oracle_job_img_sobel_hist(rgb.ctypes.data, W, H, g.ctypes.data, q.ctypes.data,
                                    s.ctypes.data, h.ctypes.data)
    return s, h


def job_mlp_ln(x_bf16: np.ndarray, w1_bf16: np.ndarray, w2_bf16: np.ndarray) -> np.ndarray:
    """fp64 out = GELU(x W1^T) W2^T + LN(x) from bf16 bit patterns."""
    from datagen import bf16_to_f32
    return mlp.mlp_ln(bf16_to_f32(x_bf16).astype(np.float64), bf16_to_f32(w1_bf16).astype(np.float64),
                      bf16_to_f32(w2_bf16).astype(np.float64))


def hotspot_params(R: int, C: int) -> dict:
    """Model parameters of an R x C hotspot grid: conductances, capacity, time step, ambient."""
    c = np.empty(6, np.float64)
    lib().oracle_hotspot_params(R, C, c.ctypes.data)
    return dict(zip(("gx", "gy", "gz", "cap", "dt", "t_amb"), (float(v) for v in c)))


def hotspot(T0: np.ndarray, P: np.ndarray, K: int) -> np.ndarray:
    """fp64 grid after K explicit steps of the hotspot model from T0 (R x C fp32) under P."""
    T0, P = _c(T0, np.float32), _c(P, np.float32)
    R, C = T0.shape
    assert P.shape == (R, C)
    T = np.empty((R, C), np.float64)
    lib().oracle_hotspot(T0.ctypes.data, P.ctypes.data, R, C, K, T.ctypes.data)
    return T
