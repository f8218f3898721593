"""set_config.sm_copies: a job graph's H2D and D2H steps as copy kernels over NVLink-C2C instead of
memcpy nodes.  Every job type, ragged byte counts (the copy kernel's tail), guard bands around the
copied regions, both completion paths; what the option refuses."""
import ctypes

import numpy as np
import pytest

from gpu_util import (S, blur_job, check_any, check_scan, check_trailers, hot_job, img_job, mlp_job, run_jobs,
                      scan_job)

pytestmark = pytest.mark.gpu


def _slot(jobs, extra=0):
    s = S()
    return max(s.set_job_slot_bytes(j.type, s.dims4(*j.dims)) for j in jobs) + extra


def test_scan_jobs_in_the_benchmarked_configuration():
    # bench.py's e2e arm: 4096 full-size scan jobs, 8 lanes x 4 slots, 4 dispatch threads, polled
    # completion, copy kernels; every job checked against the oracle
    jobs = [scan_job(k) for k in range(4096)]
    st = run_jobs(jobs, timeout_s=300, num_streams=8, num_workers=4, ring_depth=4, cb_mode=3, sm_copies=1,
                  slot_bytes=_slot(jobs))
    assert st["completed"] == 4096 and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        check_scan(j)
    check_trailers(jobs)


@pytest.mark.parametrize("cb_mode", [0, 3])
def test_every_type_and_ragged_sizes(cb_mode):
    # byte counts that are not multiples of 16 (odd n, odd image sides) exercise the tail copy
    jobs = ([blur_job(1, W=17, H=3), blur_job(2), blur_job(3, W=1, H=1), blur_job(4, W=255, H=257)] +
            [scan_job(10 + k, n=n) for k, n in enumerate([1, 3, 5, 4097, 65535, 65536, 100003])] +
            [img_job(20 + k, dims=d) for k, d in enumerate([(1, 1), (5, 3), (129, 257), (640, 480)])] +
            [mlp_job(30 + k, m=m) for k, m in enumerate([1, 77, 256])] +
            [hot_job(40, R=37, C=100, K=13), hot_job(41, R=1, C=1, K=1)])
    order = np.random.default_rng(9).permutation(len(jobs))
    jobs = [jobs[i] for i in order]
    st = run_jobs(jobs, num_streams=3, num_workers=2, ring_depth=2, cb_mode=cb_mode, sm_copies=1,
                  slot_bytes=_slot(jobs))
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        check_any(j)
    check_trailers(jobs)


def test_copy_kernels_stay_inside_the_job_regions():
    # guard bands before `in` and after in / out / scratch: the copy kernels must not touch them
    jobs = ([scan_job(50 + k, n=n) for k, n in enumerate([1, 7, 4097, 65536])] +
            [blur_job(60, W=17, H=3), blur_job(61)] + [img_job(62, dims=(5, 3)), img_job(63, dims=(129, 257))] +
            [mlp_job(64, m=77)])
    st = run_jobs(jobs, num_streams=2, num_workers=1, ring_depth=2, guards=1, sm_copies=1,
                  slot_bytes=_slot(jobs, 8192))
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        check_any(j)
    check_trailers(jobs)


def test_refused_configurations_and_buffers():
    s = S()
    for bad in (dict(io_mode=s.SET_IO_DEVICE), dict(io_mode=s.SET_IO_MAPPED), dict(batch_max=8), dict(sm_copies=2)):
        cfg = s.default_config(**dict(dict(sm_copies=1), **bad))
        ctx = ctypes.c_void_p()
        assert s.set_create_ex(ctypes.byref(cfg), ctypes.byref(ctx)) == s.SET_EINVAL
    ctx = s.create(s.default_config(sm_copies=1, slot_bytes=1 << 20))
    try:
        n = 1000
        pageable = np.zeros(8 * n, np.uint8)
        out = __import__("torch").zeros(s.set_job_out_bytes(2, s.dims4(n)) + 64, dtype=__import__("torch").uint8)
        out = out.pin_memory()
        d = s.make_desc(s.SET_JOB_SAXPY_SCAN_MAX, (n,), pageable.ctypes.data, out.data_ptr())
        assert s.set_submit(ctx, ctypes.byref(d), None) == s.SET_EINVAL  # not page-locked
        j = scan_job(70, n=n)
        d = s.make_desc(s.SET_JOB_SAXPY_SCAN_MAX, (n,), j.hin.data_ptr(), out.data_ptr() + 8)
        assert s.set_submit(ctx, ctypes.byref(d), None) == s.SET_EINVAL  # not 16-byte aligned
        assert b"sm_copies" in s.set_last_error(ctx)
        dj = scan_job(71, n=n, device=True)
        assert s.set_submit(ctx, ctypes.byref(dj.desc), None) == s.SET_EINVAL  # device memory
    finally:
        s.set_destroy(ctx)


def test_copy_kernel_rates_are_measured():
    s = S()
    for direction in (3, 4, 5):
        g = ctypes.c_double()
        s.check(s.set_copy_bandwidth(512 << 10, 8, 256, direction, ctypes.byref(g)), "set_copy_bandwidth")
        assert g.value > 1.0
