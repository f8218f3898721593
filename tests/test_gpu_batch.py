"""Batched form: queued image / MLP jobs of uneven sizes packed into one launch of the packed
persistent kernels; every job's result must match the oracle exactly as in the per-job form."""
import pytest

import datagen
from gpu_util import S, check_img, check_mlp, check_trailers, img_job, mlp_job, run_jobs, serve_jobs, check_any

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("batch_max", [4, 16])
def test_image_batches_uneven_sizes(batch_max):
    dims = [(1, 1), (5, 3), (128, 128), (700, 33), (17, 900), (256, 255), (1024, 768), (2, 2049)]
    jobs = [img_job(k, dims=dims[k % len(dims)]) for k in range(40)]
    st = run_jobs(jobs, num_streams=2, num_workers=1, ring_depth=2, slot_bytes=96 << 20, batch_max=batch_max)
    assert st["completed"] == 40 and st["failed"] == 0 and st["canary_errors"] == 0
    for j in jobs:
        check_img(j)
    check_trailers(jobs)


def test_mlp_packed_rows():
    ms = [1, 256, 7, 128, 129, 64, 3, 200]
    jobs = [mlp_job(k, m=ms[k % len(ms)]) for k in range(24)]
    st = run_jobs(jobs, num_streams=2, num_workers=1, ring_depth=2, slot_bytes=96 << 20, batch_max=8)
    assert st["completed"] == 24 and st["failed"] == 0 and st["canary_errors"] == 0
    for j in jobs:
        check_mlp(j)
    check_trailers(jobs)


def test_batches_in_the_arena_with_a_mixed_stream():
    jobs, _ = serve_jobs(1000.0, 90, img_cap=1024)
    st = run_jobs(jobs, num_streams=4, num_workers=1, ring_depth=4, slot_bytes=64 << 20, arena_bytes=1 << 30,
                  batch_max=8)
    assert st["completed"] == 90 and st["failed"] == 0 and st["canary_errors"] == 0
    for j in jobs:
        check_any(j)
    check_trailers(jobs)


@pytest.mark.parametrize("type_", [3, 4])
def test_autotuner_picks_a_candidate_and_results_stay_exact(type_):
    import ctypes
    s = S()
    if type_ == 3:
        sample = [img_job(k) for k in range(12)]
        check = check_img
    else:
        sample = [mlp_job(k) for k in range(12)]
        check = check_mlp
    ctx = s.create(s.default_config(num_streams=2, num_workers=1, ring_depth=2, slot_bytes=96 << 20, batch_max=8))
    try:
        arr = (s.set_job_desc * len(sample))(*[j.desc for j in sample])
        r = s.set_tune_result()
        s.check(s.set_autotune(ctx, type_, arr, len(sample), ctypes.byref(r)), "set_autotune", ctx)
        assert 1 <= r.batch_max <= 8 and 0 <= r.img_tile <= 2 and r.candidates >= 4 and r.jobs_per_s > 0
        assert r.jobs_per_s >= 0.95 * r.single_jobs_per_s
        first = ctypes.c_uint64()
        s.check(s.set_submit_many(ctx, arr, len(sample), ctypes.byref(first), None), "submit", ctx)
        s.check(s.set_wait_all(ctx, 60_000_000), "wait", ctx)
        for k, j in enumerate(sample):
            j.id = first.value + k
    finally:
        s.set_destroy(ctx)
    for j in sample:
        check(j)
    check_trailers(sample)


@pytest.mark.parametrize("type_", [3, 4])
def test_batched_form_in_its_bench_configuration(type_):
    # the launch configuration bench.py times for the batched form: 16 lanes x 2 slots, polled
    # completion, autotuned batches of up to 16 in an 8 GiB arena, the workload's own sizes
    import ctypes
    s = S()
    n = 160
    jobs = [img_job(k) for k in range(n)] if type_ == 3 else [mlp_job(k) for k in range(n)]
    ctx = s.create(s.default_config(num_streams=16, num_workers=1, ring_depth=2, cb_mode=3, batch_max=16,
                                    arena_bytes=8 << 30, slot_bytes=1 << 30))
    try:
        arr = (s.set_job_desc * n)(*[j.desc for j in jobs])
        r = s.set_tune_result()
        s.check(s.set_autotune(ctx, type_, arr, 64, ctypes.byref(r)), "set_autotune", ctx)
        first = ctypes.c_uint64()
        s.check(s.set_submit_many(ctx, arr, n, ctypes.byref(first), None), "submit", ctx)
        s.check(s.set_wait_all(ctx, 120_000_000), "wait", ctx)
        st = s.set_stats_t()
        s.check(s.set_stats(ctx, ctypes.byref(st)), "stats", ctx)
        assert st.completed == n and st.failed == 0 and st.canary_errors == 0
        for k, j in enumerate(jobs):
            j.id = first.value + k
    finally:
        s.set_destroy(ctx)
    for j in jobs:
        (check_img if type_ == 3 else check_mlp)(j)
    check_trailers(jobs)
