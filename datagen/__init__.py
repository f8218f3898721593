"""Seeded synthetic inputs for the five SET workloads.

Both sides of every parity check (the CPU oracle and the CUDA executor) read
the bytes produced here; this module holds none of the method's arithmetic.
All draws come from the counter-based SplitMix64 stream in ``datagen.c``.

Workloads (job payload layouts are the executor's input layouts):

* blur   (tag 1): 256x256 uint8 image, uniform 0..255.
* scan   (tag 2): x || y, two float32 vectors of n elements, uniform [-1, 1);
  per-job scalar a uniform [-2, 2).
* img    (tag 3): interleaved RGB uint8, H x W x 3; W and H drawn independently,
  log-uniform on [128, 2048].
* mlp    (tag 4): m x 1024 bf16 rows, m uniform on 1..256, x ~ N(0, 1);
  shared weights W1 [4096, 1024] ~ N(0, 1/1024), W2 [1024, 4096] ~ N(0, 1/4096),
  both stored out_features x in_features (h = x W1^T).
* serve  (tag 5): Poisson arrivals (exponential gaps) and a 40/40/20 type mix.
* hot    (tag 6): hotspot grid, T0 || P, two float32 R x C maps: T0 uniform [80, 90)
  degrees, P uniform [0, 1e-3) watts per cell (512 x 512 cells, 64 steps in the
  workload).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

MASTER_SEED = 2606055495
TAG_BLUR, TAG_SCAN, TAG_IMG, TAG_MLP, TAG_SERVE, TAG_HOT = 1, 2, 3, 4, 5, 6
TAG_W1, TAG_W2 = 0x41, 0x42

BLUR_SIDE = 256
SCAN_N = 65536
IMG_SIDE_MIN, IMG_SIDE_MAX = 128, 2048
MLP_D, MLP_F, MLP_M_MAX = 1024, 4096, 256
HOT_SIDE, HOT_STEPS = 512, 64
HOT_T0 = (80.0, 90.0)
HOT_P = (0.0, 1e-3)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libdatagen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile libdatagen.so beside this file (gcc, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "datagen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u64, u32, sz, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int
            vp, dbl = ctypes.c_void_p, ctypes.c_double
            L.dg_rand.argtypes, L.dg_rand.restype = [u64, u64], u64
            L.dg_job_seed.argtypes, L.dg_job_seed.restype = [u64, u32, u64], u64
            L.dg_fill_u8.argtypes, L.dg_fill_u8.restype = [u64, u64, vp, sz], None
            L.dg_fill_unif_sym_f32.argtypes, L.dg_fill_unif_sym_f32.restype = [u64, u64, i32, vp, sz], None
            L.dg_unif_sym_f32.argtypes, L.dg_unif_sym_f32.restype = [u64, u64, i32], ctypes.c_float
            L.dg_unif01.argtypes, L.dg_unif01.restype = [u64, u64], dbl
            L.dg_fill_normal_bf16.argtypes, L.dg_fill_normal_bf16.restype = [u64, u64, dbl, vp, sz], None
            L.dg_logunif_side.argtypes, L.dg_logunif_side.restype = [u64, u64, i32, i32], i32
            L.dg_exp_gap.argtypes, L.dg_exp_gap.restype = [u64, u64, dbl], dbl
            L.dg_fill_unif_range_f32.argtypes = [u64, u64, dbl, dbl, vp, sz]
            L.dg_fill_unif_range_f32.restype = None
            _lib = L
    return _lib


def _out(out, shape, dtype):
    if out is None:
        return np.empty(shape, dtype=dtype)
    assert out.dtype == dtype and out.size == int(np.prod(shape)) and out.flags.c_contiguous
    return out.reshape(shape)


def rand(seed: int, i: int) -> int:
    return int(lib().dg_rand(seed, i))


def job_seed(tag: int, job: int, master: int = MASTER_SEED) -> int:
    return int(lib().dg_job_seed(master, tag, job))


def blur_job(j: int, out=None, master: int = MASTER_SEED) -> np.ndarray:
    """256x256 uint8 image of blur job j."""
    o = _out(out, (BLUR_SIDE, BLUR_SIDE), np.uint8)
    lib().dg_fill_u8(job_seed(TAG_BLUR, j, master), 0, o.ctypes.data, o.size)
    return o


def scan_scalar(j: int, n: int = SCAN_N, master: int = MASTER_SEED) -> float:
    """Per-job saxpy scalar a, uniform [-2, 2), drawn at stream index 2n."""
    return float(lib().dg_unif_sym_f32(job_seed(TAG_SCAN, j, master), 2 * n, 1))


def scan_job(j: int, n: int = SCAN_N, out=None, master: int = MASTER_SEED):
    """(a, xy) for scan job j; xy is x (n floats) followed by y (n floats)."""
    o = _out(out, (2 * n,), np.float32)
    lib().dg_fill_unif_sym_f32(job_seed(TAG_SCAN, j, master), 0, 0, o.ctypes.data, o.size)
    return scan_scalar(j, n, master), o


def img_dims(j: int, master: int = MASTER_SEED):
    """(W, H) of image job j, independently log-uniform on [128, 2048]."""
    s = job_seed(TAG_IMG, j, master)
    L = lib()
    return (int(L.dg_logunif_side(s, 0, IMG_SIDE_MIN, IMG_SIDE_MAX)),
            int(L.dg_logunif_side(s, 1, IMG_SIDE_MIN, IMG_SIDE_MAX)))


def img_job(j: int, out=None, master: int = MASTER_SEED, dims=None) -> np.ndarray:
    """Interleaved RGB uint8 image (H, W, 3) of image job j (dims override W, H)."""
    W, H = dims if dims is not None else img_dims(j, master)
    o = _out(out, (H, W, 3), np.uint8)
    lib().dg_fill_u8(job_seed(TAG_IMG, j, master), 2, o.ctypes.data, o.size)
    return o


def mlp_rows(j: int, master: int = MASTER_SEED) -> int:
    """m of MLP job j, uniform on 1..256 (top byte of draw 0, plus one)."""
    return 1 + (rand(job_seed(TAG_MLP, j, master), 0) >> 56)


def mlp_job(j: int, out=None, master: int = MASTER_SEED, m=None) -> np.ndarray:
    """x of MLP job j as bf16 bit patterns (uint16), shape (m, 1024)."""
    m = mlp_rows(j, master) if m is None else m
    o = _out(out, (m, MLP_D), np.uint16)
    lib().dg_fill_normal_bf16(job_seed(TAG_MLP, j, master), 1, 1.0, o.ctypes.data, o.size)
    return o


def mlp_weights(master: int = MASTER_SEED, d: int = MLP_D, f: int = MLP_F):
    """(W1 [f, d], W2 [d, f]) as bf16 bit patterns; N(0, 1/fan_in)."""
    w1 = np.empty((f, d), np.uint16)
    w2 = np.empty((d, f), np.uint16)
    L = lib()
    L.dg_fill_normal_bf16(job_seed(TAG_W1, 0, master), 0, 1.0 / np.sqrt(d), w1.ctypes.data, w1.size)
    L.dg_fill_normal_bf16(job_seed(TAG_W2, 0, master), 0, 1.0 / np.sqrt(f), w2.ctypes.data, w2.size)
    return w1, w2


def bf16_to_f32(b: np.ndarray) -> np.ndarray:
    """Widen bf16 bit patterns to float32 (exact)."""
    return (b.astype(np.uint32) << 16).view(np.float32)


def hot_job(j: int, R: int = HOT_SIDE, C: int = HOT_SIDE, out=None, master: int = MASTER_SEED) -> np.ndarray:
    """T0 (R x C) followed by P (R x C), float32, of hotspot job j."""
    o = _out(out, (2 * R * C,), np.float32)
    s = job_seed(TAG_HOT, j, master)
    L = lib()
    L.dg_fill_unif_range_f32(s, 0, HOT_T0[0], HOT_T0[1], o.ctypes.data, R * C)
    L.dg_fill_unif_range_f32(s, R * C, HOT_P[0], HOT_P[1], o[R * C:].ctypes.data, R * C)
    return o


SERVE_MIX = ((1, 0.4), (3, 0.4), (4, 0.2))  # (workload tag, share)


def serve_trace(lam: float, n: int, master: int = MASTER_SEED):
    """Poisson arrival trace for rate lam (jobs/s): (arrival seconds, workload tags, job ids).

    Gaps are exponential draws of the per-rate stream; the type of arrival i is
    chosen by a second uniform draw against the 40/40/20 mix.  Job ids index the
    per-workload generators above and are distinct per trace.
    """
    s = job_seed(TAG_SERVE, int(lam), master)
    L = lib()
    gaps = np.array([L.dg_exp_gap(s, 2 * i, lam) for i in range(n)])
    u = np.array([L.dg_unif01(s, 2 * i + 1) for i in range(n)])
    edges = np.cumsum([p for _, p in SERVE_MIX])
    kinds = np.array([SERVE_MIX[int(np.searchsorted(edges, x, side="right"))][0] for x in u])
    ids = (np.arange(n) + (int(lam) << 20)).astype(np.int64)
    return np.cumsum(gaps), kinds, ids
