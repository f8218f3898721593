"""Helpers shared by the GPU tests: pinned buffers, job building, running jobs through the executor."""
from __future__ import annotations

import ctypes

import numpy as np

import datagen


def S():
    import paper_2606_05495_gb300 as mod
    return mod


def torch():
    import torch as t
    return t


class Job:
    """One job with its pinned input/output buffers (kept alive until checked)."""

    def __init__(self, type_, dims, payload: np.ndarray, scalar=0.0, shared=(None, None), device=False):
        s, t = S(), torch()
        self.type, self.dims, self.scalar, self.payload = type_, tuple(dims), scalar, payload
        raw = np.ascontiguousarray(payload).view(np.uint8).ravel()
        ob = s.set_job_out_bytes(type_, s.dims4(*dims))
        assert raw.size == s.set_job_in_bytes(type_, s.dims4(*dims)) and ob > 0
        if device:
            self.hin = t.from_numpy(raw.copy()).cuda()
            self.hout = t.zeros(ob, dtype=t.uint8, device="cuda")
        else:
            self.hin = t.from_numpy(raw.copy()).pin_memory()
            self.hout = t.full((ob,), 0xAB, dtype=t.uint8).pin_memory()
        self.status = ctypes.c_int32(99)
        self.desc = s.make_desc(type_, dims, self.hin.data_ptr(), self.hout.data_ptr(), scalar=scalar,
                                shared=shared, status=ctypes.pointer(self.status))
        self.id = None

    def out(self) -> np.ndarray:
        return self.hout.cpu().numpy() if self.hout.is_cuda else self.hout.numpy()

    def trailer(self):
        o = self.out()
        t = o[-16:]
        return int(t[:8].view(np.uint64)[0]), int(t[8:12].view(np.uint32)[0]), int(t[12:16].view(np.uint32)[0])


def run_jobs(jobs, timeout_s=120, **cfg):
    """Submits every job (set_submit_many), waits, returns the context's stats dict."""
    s = S()
    ctx = s.create(s.default_config(**cfg))
    try:
        arr = (s.set_job_desc * len(jobs))(*[j.desc for j in jobs])
        first = ctypes.c_uint64()
        s.check(s.set_submit_many(ctx, arr, len(jobs), ctypes.byref(first), None), "set_submit_many", ctx)
        s.check(s.set_wait_all(ctx, int(timeout_s * 1e6)), "set_wait_all", ctx)
        for k, j in enumerate(jobs):
            j.id = first.value + k
        st = s.set_stats_t()
        s.check(s.set_stats(ctx, ctypes.byref(st)), "set_stats", ctx)
        return st.as_dict()
    finally:
        s.set_destroy(ctx)


def check_trailers(jobs, io_host=True):
    s = S()
    for j in jobs:
        jid, gen, word = j.trailer()
        assert jid == j.id, (jid, j.id)
        assert word == (s.SET_TRAILER_MAGIC << 16), hex(word)
        if io_host:
            assert j.status.value == s.SET_OK, j.status.value


# ---- per-type oracle comparisons ----

def blur_job(j, W=256, H=256, **kw):
    img = datagen.blur_job(j) if (W, H) == (256, 256) else np.random.default_rng(j).integers(
        0, 256, (H, W), dtype=np.uint8)
    return Job(S().SET_JOB_BLUR_HIST, (W, H), img, **kw)


def check_blur(job):
    import oracle
    W, H = job.dims
    b, h = oracle.job_blur_hist(job.payload.reshape(H, W))
    o = job.out()
    n = W * H
    off = (n + 15) & ~15
    assert np.array_equal(o[:n].reshape(H, W), b), f"blurred image mismatch at {W}x{H}"
    assert not o[n:off].any(), "pad bytes not zero"
    assert np.array_equal(o[off:off + 1024].view(np.uint32), h), f"histogram mismatch at {W}x{H}"


def scan_job(j, n=datagen.SCAN_N, **kw):
    a, xy = datagen.scan_job(j, n=n)
    return Job(S().SET_JOB_SAXPY_SCAN_MAX, (n,), xy, scalar=a, **kw)


SCAN_RTOL = 1e-5  # |S_gpu - S| <= 1e-5 * sum_{j<i} |z_j|  (fp32 vs the fp64 oracle)


def check_scan(job):
    import oracle
    n = job.dims[0]
    xy = job.payload
    z, Sref, A, m = oracle.job_saxpy_scan_max(job.scalar, xy[:n], xy[n:])
    f = job.out()[:8 * n + 16].view(np.float32)
    assert np.array_equal(f[:n], z), "z is not bit-exact"
    err = np.abs(f[n:2 * n].astype(np.float64) - Sref)
    assert np.all(err <= SCAN_RTOL * A), f"scan error {np.max(err / np.maximum(A, 1e-300))} x A"
    assert f[n] == 0.0 if n else True  # S_0 is exactly 0
    assert abs(float(f[2 * n]) - m) <= SCAN_RTOL * float(A.max()), (float(f[2 * n]), m)
    assert not f[2 * n + 1:2 * n + 4].any(), "pad after m not zero"


def img_job(j, dims=None, **kw):
    rgb = datagen.img_job(j, dims=dims)
    H, W, _ = rgb.shape
    return Job(S().SET_JOB_IMG_SOBEL_HIST, (W, H), rgb, **kw)


def check_img(job):
    import oracle
    W, H = job.dims
    s_ref, h_ref = oracle.job_img_sobel_hist(job.payload.reshape(H, W, 3))
    o = job.out()
    n = W * H
    off = (n + 15) & ~15
    got = o[:n].reshape(H, W)
    if not np.array_equal(got, s_ref):
        bad = np.argwhere(got != s_ref)
        raise AssertionError(f"Sobel image mismatch at {W}x{H}: {len(bad)} px, first {bad[:5].tolist()}")
    assert not o[n:off].any(), "pad bytes not zero"
    assert np.array_equal(o[off:off + 1024].view(np.uint32), h_ref), f"histogram mismatch at {W}x{H}"


_WEIGHTS = {}


def mlp_weights_dev():
    """(W1, W2) bf16 device tensors (kept for the session) and their host bit patterns."""
    if "w" not in _WEIGHTS:
        t = torch()
        w1, w2 = datagen.mlp_weights()
        _WEIGHTS["w"] = (t.from_numpy(w1.view(np.int16)).cuda(), t.from_numpy(w2.view(np.int16)).cuda(), w1, w2)
    return _WEIGHTS["w"]


def mlp_job(j, m=None, **kw):
    d1, d2, _, _ = mlp_weights_dev()
    x = datagen.mlp_job(j, m=m)
    return Job(S().SET_JOB_MLP_LN, (x.shape[0],), x, shared=(d1.data_ptr(), d2.data_ptr()), **kw)


MLP_RTOL = 2e-2  # |out - ref| <= 2e-2 * max(|ref|, rms(ref of the job))


def check_mlp(job):
    import oracle
    _, _, w1, w2 = mlp_weights_dev()
    m = job.dims[0]
    ref = oracle.job_mlp_ln(job.payload.reshape(m, 1024), w1, w2)
    got = job.out()[:m * 4096].view(np.float32).reshape(m, 1024).astype(np.float64)
    assert np.isfinite(got).all(), "non-finite output"
    rms = float(np.sqrt(np.mean(ref * ref)))
    err = np.abs(got - ref)
    bound = MLP_RTOL * np.maximum(np.abs(ref), rms)
    worst = float(np.max(err / bound))
    assert worst <= 1.0, f"m={m}: worst error {worst:.3f} of the bound; max abs err {err.max():.3e}"
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert rel < 1e-2, f"m={m}: norm-wise relative error {rel:.3e}"
    return rel


def serve_jobs(lam, n, img_cap=None):
    """Jobs and arrival offsets (ns) of a Poisson trace mixing blur / image / MLP jobs 40/40/20.
    img_cap bounds image sides (keeps the oracle quick in tests)."""
    t, kinds, ids = datagen.serve_trace(lam, n)
    jobs = []
    for kind, j in zip(kinds, ids):
        if kind == 1:
            jobs.append(blur_job(int(j)))
        elif kind == 3:
            W, H = datagen.img_dims(int(j))
            if img_cap:
                W, H = min(W, img_cap), min(H, img_cap)
            jobs.append(img_job(int(j), dims=(W, H)))
        else:
            jobs.append(mlp_job(int(j)))
    return jobs, (t * 1e9).astype(np.uint64)


def hot_job(j, R=datagen.HOT_SIDE, C=datagen.HOT_SIDE, K=datagen.HOT_STEPS, **kw):
    x = datagen.hot_job(j, R, C)
    return Job(S().SET_JOB_HOTSPOT, (C, R, K), x, **kw)


HOT_RTOL = 1e-5  # |T_gpu - T| <= 1e-5 |T| per cell (fp32 steps vs the fp64 oracle)


def check_hot(job):
    import oracle
    C, R, K = job.dims
    x = job.payload
    ref = oracle.hotspot(x[:R * C].reshape(R, C), x[R * C:].reshape(R, C), K)
    o = job.out()
    got = o[:4 * R * C].view(np.float32).reshape(R, C).astype(np.float64)
    assert np.isfinite(got).all(), "non-finite temperature"
    rel = np.abs(got - ref) / np.abs(ref)
    worst = float(rel.max())
    assert worst <= HOT_RTOL, f"{C}x{R}, K={K}: worst relative error {worst:.3e} at {np.unravel_index(rel.argmax(), rel.shape)}"
    off = (4 * R * C + 15) & ~15
    assert not o[4 * R * C:off].any(), "pad bytes not zero"
    return worst


def check_any(job):
    {1: check_blur, 2: check_scan, 3: check_img, 4: check_mlp, 5: check_hot}[job.type](job)
