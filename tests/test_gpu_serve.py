"""Serving form: Poisson arrivals of mixed jobs (blur / image / MLP, 40/40/20), admission by free
arena memory, continuous batching.  Each job's result in the mix must equal its result alone."""
import ctypes

import numpy as np
import pytest

from gpu_util import S, check_any, check_trailers, serve_jobs, run_jobs

pytestmark = pytest.mark.gpu


def _serve(jobs, arrivals, mode, **cfg):
    s = S()
    ctx = s.create(s.default_config(**cfg))
    try:
        arr = (s.set_job_desc * len(jobs))(*[j.desc for j in jobs])
        ts = (ctypes.c_uint64 * len(jobs))(*[int(a) for a in arrivals])
        st = s.set_stats_t()
        s.check(s.set_serve(ctx, mode, arr, ts, len(jobs), ctypes.byref(st)), "set_serve", ctx)
        return st.as_dict()
    finally:
        s.set_destroy(ctx)


ARENA_CFG = dict(num_streams=6, num_workers=1, ring_depth=4, slot_bytes=64 << 20, arena_bytes=1 << 30)


def test_serving_mix_equals_alone_and_oracle():
    jobs, arrivals = serve_jobs(4000.0, 150, img_cap=1024)
    st = _serve(jobs, arrivals, S().SET_SERVE_SET, **ARENA_CFG)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    assert 0 < st["p50_us"] <= st["p99_us"]
    mixed = [j.out().copy() for j in jobs]
    for j in jobs:
        check_any(j)
    # alone: one job at a time on an idle context, same kernels
    s = S()
    ctx = s.create(s.default_config(num_streams=1, num_workers=1, slot_bytes=64 << 20, arena_bytes=256 << 20))
    try:
        for k, j in enumerate(jobs[:60]):
            j.hout.fill_(0)
            s.check(s.set_submit(ctx, ctypes.byref(j.desc), None), "set_submit", ctx)
            s.check(s.set_wait_all(ctx, 30_000_000), "set_wait_all", ctx)
            alone = j.out()
            n = j.desc.out_bytes - 16  # the trailer differs (job id, slot generation)
            if j.type == 4:
                a = alone[:n].view(np.float32)
                b = mixed[k][:n].view(np.float32)
                assert np.allclose(a, b, rtol=0, atol=2e-2 * max(1.0, float(np.abs(a).max()))), k
            else:
                assert np.array_equal(alone[:n], mixed[k][:n]), k
    finally:
        s.set_destroy(ctx)


def test_serving_polled_completion():
    jobs, arrivals = serve_jobs(8000.0, 120, img_cap=1024)
    st = _serve(jobs, arrivals, S().SET_SERVE_SET, cb_mode=3, **ARENA_CFG)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    assert 0 < st["mean_queue_us"] and st["mean_queue_us"] + st["mean_service_us"] >= 0.5 * st["p50_us"]
    for j in jobs:
        check_any(j)


def test_serving_launch_at_submit():
    # the request loop binds and launches each arrival itself when a slot and its memory are free
    jobs, arrivals = serve_jobs(8000.0, 120, img_cap=1024)
    st = _serve(jobs, arrivals, S().SET_SERVE_SET, cb_mode=3, bind_at_submit=2, **ARENA_CFG)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        check_any(j)


def test_serving_batch_sync_baseline_same_arrivals():
    jobs, arrivals = serve_jobs(4000.0, 80, img_cap=1024)
    st = _serve(jobs, arrivals, S().SET_SERVE_BATCH_SYNC, **ARENA_CFG)
    assert st["completed"] == len(jobs) and st["p99_us"] > 0
    for j in jobs:
        check_any(j)


def test_arena_admission_waits_for_memory():
    # a 20 MiB arena holds a 16 MiB buddy range: two 1024x1024 image jobs (8 MiB blocks) at a time
    from gpu_util import blur_job, img_job
    jobs = [blur_job(k) for k in range(6)] + [img_job(900 + k, dims=(1024, 1024)) for k in range(6)]
    arrivals = (np.arange(len(jobs), dtype=np.uint64) * 2000)  # one every 2 us
    st = _serve(jobs, arrivals, S().SET_SERVE_SET, num_streams=4, num_workers=1, ring_depth=2, slot_bytes=16 << 20,
                arena_bytes=20 << 20)
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["mem_waits"] > 0 and st["arena_peak_bytes"] <= 16 << 20
    for j in jobs:
        check_any(j)
