"""GPU parity of the blur and scan jobs through the C ABI (executor and direct launches)."""
import ctypes

import numpy as np
import pytest

from gpu_util import S, blur_job, check_blur, check_scan, check_trailers, run_jobs, scan_job, torch

pytestmark = pytest.mark.gpu


def test_blur_config_64_jobs_2_streams():
    jobs = [blur_job(j) for j in range(64)]
    st = run_jobs(jobs, num_streams=2, num_workers=2, slot_bytes=1 << 20)
    assert st["completed"] == 64 and st["failed"] == 0 and st["canary_errors"] == 0
    for j in jobs:
        check_blur(j)
    check_trailers(jobs)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (16, 16), (17, 3), (33, 7), (300, 9), (255, 257),
                                 (2048, 40), (64, 1000)])
def test_blur_edge_sizes(W, H):
    jobs = [blur_job(k, W=W, H=H) for k in range(3)]
    st = run_jobs(jobs, num_streams=2, num_workers=1, slot_bytes=4 << 20)
    assert st["failed"] == 0
    for j in jobs:
        check_blur(j)
    check_trailers(jobs)


def test_scan_config_4096_jobs_8_streams_stealing():
    jobs = [scan_job(j) for j in range(4096)]
    st = run_jobs(jobs, timeout_s=300, num_streams=8, num_workers=8, ring_depth=2,
                  slot_bytes=S().set_job_slot_bytes(2, S().dims4(65536)))
    assert st["completed"] == 4096 and st["failed"] == 0 and st["canary_errors"] == 0
    for j in jobs:
        check_scan(j)
    check_trailers(jobs)


def test_scan_headline_launch_configuration():
    # the configuration bench.py times: 4096 full-size jobs, 16 lanes x 4 slots, 4 dispatch threads,
    # polled completion, stealing; every job checked against the oracle
    jobs = [scan_job(j) for j in range(4096)]
    st = run_jobs(jobs, timeout_s=300, num_streams=16, num_workers=4, ring_depth=4, cb_mode=3,
                  slot_bytes=S().set_job_slot_bytes(2, S().dims4(65536)))
    assert st["completed"] == 4096 and st["failed"] == 0 and st["canary_errors"] == 0
    for j in jobs:
        check_scan(j)
    check_trailers(jobs)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 4095, 4096, 4097, 65537, 100003, 1 << 20])
def test_scan_edge_sizes(n):
    jobs = [scan_job(k, n=n) for k in range(3)]
    st = run_jobs(jobs, num_streams=2, num_workers=2, slot_bytes=max(1 << 20, 20 * n + 65536))
    assert st["failed"] == 0
    for j in jobs:
        check_scan(j)
    check_trailers(jobs)


def test_mixed_types_share_slots_without_stealing():
    jobs = []
    for k in range(40):
        jobs.append(blur_job(k) if k % 2 else scan_job(k, n=65536 - 7 * k))
    st = run_jobs(jobs, num_streams=3, num_workers=2, slot_bytes=2 << 20, steal=0)
    assert st["failed"] == 0 and st["steals"] == 0
    for j in jobs:
        (check_blur if j.type == S().SET_JOB_BLUR_HIST else check_scan)(j)
    check_trailers(jobs)


def test_device_io_mode():
    jobs = [scan_job(k, device=True) for k in range(16)] + [blur_job(k, device=True) for k in range(16)]
    st = run_jobs(jobs, num_streams=4, num_workers=2, slot_bytes=2 << 20, io_mode=S().SET_IO_DEVICE)
    assert st["failed"] == 0 and st["completed"] == 32
    for j in jobs:
        (check_blur if j.type == S().SET_JOB_BLUR_HIST else check_scan)(j)
    check_trailers(jobs, io_host=False)


def test_direct_launch_reuses_scan_scratch_across_sizes():
    s, t = S(), torch()
    ns = [65536, 1, 4097, 300000, 4096, 7]
    scratch = t.zeros(max(s.set_job_scratch_bytes(2, s.dims4(n)) for n in ns), dtype=t.uint8, device="cuda")
    stream = t.cuda.current_stream().cuda_stream
    for k, n in enumerate(ns):
        j = scan_job(k, n=n, device=True)
        st = s.set_launch_job(ctypes.byref(j.desc), j.hin.data_ptr(), j.hout.data_ptr(), scratch.data_ptr(), 1000 + k, 0,
                              stream)
        assert st == 0
        t.cuda.synchronize()
        check_scan(j)
        assert j.trailer()[0] == 1000 + k


@pytest.mark.parametrize("kind", [1, 2])
def test_baselines_compute_the_same_results(kind):
    s = S()
    jobs = [scan_job(k) for k in range(10)] + [blur_job(k) for k in range(10)]
    ctx = s.create(s.default_config(num_streams=4, num_workers=2, slot_bytes=2 << 20))
    try:
        arr = (s.set_job_desc * len(jobs))(*[j.desc for j in jobs])
        st = s.set_stats_t()
        s.check(s.set_run_baseline(ctx, kind, arr, len(jobs), ctypes.byref(st)), "set_run_baseline", ctx)
        assert st.completed == len(jobs) and st.jobs_per_s > 0
    finally:
        s.set_destroy(ctx)
    for j in jobs:
        (check_blur if j.type == s.SET_JOB_BLUR_HIST else check_scan)(j)


@pytest.mark.parametrize("cb_mode", [0, 1, 2, 3])
def test_callback_modes_and_baseline_reuse(cb_mode):
    s = S()
    jobs = [scan_job(k, n=20000 + k) for k in range(120)]
    ctx = s.create(s.default_config(num_streams=4, num_workers=1, slot_bytes=1 << 20, cb_mode=cb_mode))
    try:
        # a baseline first: it reuses the slots' graphs, whose completion path must stay quiet
        arr = (s.set_job_desc * 8)(*[j.desc for j in jobs[:8]])
        st = s.set_stats_t()
        s.check(s.set_run_baseline(ctx, s.SET_BASE_BATCH_SYNC, arr, 8, ctypes.byref(st)), "baseline", ctx)
        arr = (s.set_job_desc * len(jobs))(*[j.desc for j in jobs])
        first = ctypes.c_uint64()
        s.check(s.set_submit_many(ctx, arr, len(jobs), ctypes.byref(first), None), "submit", ctx)
        s.check(s.set_wait_all(ctx, 60_000_000), "wait", ctx)
        s.check(s.set_stats(ctx, ctypes.byref(st)), "stats", ctx)
        assert st.completed == len(jobs) and st.failed == 0 and st.canary_errors == 0
        for k, j in enumerate(jobs):
            j.id = first.value + k
    finally:
        s.set_destroy(ctx)
    for j in jobs:
        check_scan(j)
    check_trailers(jobs)


@pytest.mark.parametrize("cb_every", [1, 3])
def test_polled_completion_destroy_with_jobs_in_flight(cb_every):
    # cb_mode 3: the completion thread must hand back every job, also when the context is
    # destroyed right after the last submit
    s = S()
    jobs = [scan_job(500 + k, n=30000 + 7 * k) for k in range(96)]
    ctx = s.create(s.default_config(num_streams=3, num_workers=1, ring_depth=2, slot_bytes=1 << 20, cb_mode=3,
                                    cb_every=cb_every))
    arr = (s.set_job_desc * len(jobs))(*[j.desc for j in jobs])
    first = ctypes.c_uint64()
    try:
        s.check(s.set_submit_many(ctx, arr, len(jobs), ctypes.byref(first), None), "submit", ctx)
    finally:
        s.set_destroy(ctx)
    for k, j in enumerate(jobs):
        j.id = first.value + k
        assert j.status.value == 0, (k, j.status.value)
        check_scan(j)
    check_trailers(jobs)


@pytest.mark.parametrize("kind", ["blur", "scan", "img"])
def test_smallest_job_in_a_slot_sized_for_it(kind):
    # the graph template of every type fits a slot sized by set_job_slot_bytes for its smallest job
    from gpu_util import check_img, img_job
    s = S()
    job = {"blur": lambda: blur_job(1, W=1, H=1), "scan": lambda: scan_job(2, n=1),
           "img": lambda: img_job(3, dims=(1, 1))}[kind]()
    slot = s.set_job_slot_bytes(job.type, s.dims4(*job.dims))
    st = run_jobs([job], num_streams=1, num_workers=1, ring_depth=1, slot_bytes=slot)
    assert st["completed"] == 1 and st["failed"] == 0
    {"blur": check_blur, "scan": check_scan, "img": check_img}[kind](job)
    check_trailers([job])


@pytest.mark.parametrize("cb_mode,workers", [(0, 1), (3, 2)])
def test_bind_at_submit(cb_mode, workers):
    # UpdateGraphParams on the submitting thread, dispatch only launches
    jobs = [scan_job(800 + k, n=40000 + 13 * k) for k in range(60)] + [blur_job(900 + k) for k in range(40)]
    st = run_jobs(jobs, num_streams=4, num_workers=workers, ring_depth=2, slot_bytes=1 << 20, cb_mode=cb_mode,
                  bind_at_submit=1)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        (check_blur if j.type == S().SET_JOB_BLUR_HIST else check_scan)(j)
    check_trailers(jobs)


def test_bounded_device_wait_reports_and_context_survives():
    # failure detection without a GPU fault: a scan tile that never publishes makes the next tile's
    # look-back (and the final max gather) wait until its bound runs out; the job completes with
    # SET_EDEVICE (trailer error bit), its neighbours on the same slot are unaffected
    s = S()
    jobs = [scan_job(1000 + k, n=65536) for k in range(5)]
    jobs[2].desc.flags = s.SET_F_TEST_STALL
    slot = s.set_job_slot_bytes(s.SET_JOB_SAXPY_SCAN_MAX, s.dims4(65536))
    st = run_jobs(jobs, num_streams=1, num_workers=1, ring_depth=1, slot_bytes=slot, cb_mode=3)
    assert st["completed"] == 5 and st["failed"] == 1 and st["canary_errors"] == 0, st
    assert jobs[2].status.value == s.SET_EDEVICE
    _, _, word = jobs[2].trailer()
    assert word == (s.SET_TRAILER_MAGIC << 16) | s.SET_DEVERR_WAIT, hex(word)
    for k in (0, 1, 3, 4):
        assert jobs[k].status.value == s.SET_OK
        check_scan(jobs[k])


def test_stats_carry_the_traced_kernel_gap():
    import math
    s = S()
    jobs = [scan_job(1200 + k, n=65536) for k in range(64)]
    slot = s.set_job_slot_bytes(s.SET_JOB_SAXPY_SCAN_MAX, s.dims4(65536))
    ctx = s.create(s.default_config(num_streams=4, num_workers=2, ring_depth=2, slot_bytes=slot, cb_mode=3))
    try:
        st = s.set_stats_t()
        s.check(s.set_stats(ctx, ctypes.byref(st)), "stats", ctx)
        assert math.isnan(st.mean_kernel_gap_us)
        arr = (s.set_job_desc * len(jobs))(*[j.desc for j in jobs])
        tr = s.set_trace_summary()
        if s.set_trace_start() != s.SET_OK:
            pytest.skip("CUPTI activity tracing unavailable")
        s.check(s.set_submit_many(ctx, arr, len(jobs), None, None), "submit", ctx)
        s.check(s.set_wait_all(ctx, 60_000_000), "wait", ctx)
        s.check(s.set_trace_stop(ctypes.byref(tr)), "trace stop")
        s.check(s.set_stats(ctx, ctypes.byref(st)), "stats", ctx)
        assert tr.kernels == len(jobs) and st.mean_kernel_gap_us == tr.mean_kernel_gap_us >= 0
        s.check(s.set_reset_stats(ctx), "reset", ctx)
        s.check(s.set_stats(ctx, ctypes.byref(st)), "stats", ctx)
        assert math.isnan(st.mean_kernel_gap_us)  # the trace began before the reset
    finally:
        s.set_destroy(ctx)
    for j in jobs:
        check_scan(j)
