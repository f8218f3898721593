"""SET_IO_DEVICE_INPLACE: the stage kernels read and write the jobs' device buffers in place (graphs
without copy nodes); results must equal the oracle exactly as with copy nodes."""
import ctypes

import numpy as np
import pytest

from gpu_util import (S, blur_job, check_blur, check_hot, check_img, check_scan, check_trailers, hot_job, img_job,
                      mlp_job, run_jobs, scan_job)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cb_mode", [0, 3])
def test_inplace_all_copyless_types(cb_mode):
    s = S()
    jobs = ([blur_job(k, device=True) for k in range(4)] + [blur_job(50, W=17, H=3, device=True)] +
            [scan_job(100 + k, n=65536 - 999 * k, device=True) for k in range(4)] +
            [scan_job(110, n=1, device=True), scan_job(111, n=4097, device=True)] +
            [img_job(200 + k, dims=d, device=True) for k, d in enumerate([(300, 200), (129, 1), (1, 70), (640, 480)])] +
            [hot_job(300, R=37, C=100, K=13, device=True), hot_job(301, R=512, C=512, K=64, device=True)])
    order = np.random.default_rng(3).permutation(len(jobs))
    jobs = [jobs[i] for i in order]
    slot = max(s.set_job_slot_bytes(j.type, s.dims4(*j.dims)) for j in jobs)
    st = run_jobs(jobs, num_streams=3, num_workers=2, ring_depth=2, slot_bytes=slot,
                  io_mode=s.SET_IO_DEVICE_INPLACE, cb_mode=cb_mode)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        {1: check_blur, 2: check_scan, 3: check_img, 5: check_hot}[j.type](j)
    check_trailers(jobs, io_host=False)


def test_inplace_headline_scan_configuration():
    # bench.py's value arm: 4096 full-size scan jobs in HBM, 8 lanes x 4 slots, 4 dispatch threads,
    # polled completion, read and written in place
    jobs = [scan_job(k, device=True) for k in range(4096)]
    s = S()
    st = run_jobs(jobs, timeout_s=300, num_streams=8, num_workers=4, ring_depth=4, cb_mode=3,
                  io_mode=s.SET_IO_DEVICE_INPLACE, slot_bytes=s.set_job_slot_bytes(2, s.dims4(65536)))
    assert st["completed"] == 4096 and st["failed"] == 0, st
    for j in jobs:
        check_scan(j)
    check_trailers(jobs, io_host=False)


def test_inplace_refusals():
    s = S()
    cfg = s.default_config(num_streams=1, num_workers=1, slot_bytes=1 << 20, io_mode=s.SET_IO_DEVICE_INPLACE,
                           batch_max=4)
    ctx = ctypes.c_void_p()
    assert s.set_create_ex(ctypes.byref(cfg), ctypes.byref(ctx)) == s.SET_EINVAL
    slot = s.set_job_slot_bytes(s.SET_JOB_MLP_LN, s.dims4(16))
    ctx = s.create(s.default_config(num_streams=1, num_workers=1, slot_bytes=slot, io_mode=s.SET_IO_DEVICE_INPLACE))
    try:
        m = mlp_job(5, m=16, device=True)
        assert s.set_submit(ctx, ctypes.byref(m.desc), None) == s.SET_EINVAL
        host = scan_job(6, n=1000)  # page-locked host buffers
        assert s.set_submit(ctx, ctypes.byref(host.desc), None) == s.SET_EINVAL
        dev = scan_job(7, n=1000, device=True)
        d = s.make_desc(s.SET_JOB_SAXPY_SCAN_MAX, (1000,), dev.hin.data_ptr() + 4, dev.hout.data_ptr())
        assert s.set_submit(ctx, ctypes.byref(d), None) == s.SET_EINVAL  # not 16-byte aligned
        assert b"in-place" in s.set_last_error(ctx)
        arr = (s.set_job_desc * 1)(dev.desc)
        st = s.set_stats_t()
        assert s.set_run_baseline(ctx, s.SET_BASE_BATCH_SYNC, arr, 1, ctypes.byref(st)) == s.SET_EINVAL
    finally:
        s.set_destroy(ctx)
