"""SET_IO_MAPPED: the stage kernels read and write the jobs' page-locked host buffers directly
(no copy nodes); results must equal the oracle exactly as with copy nodes."""
import ctypes

import numpy as np
import pytest

from gpu_util import (S, blur_job, check_blur, check_hot, check_img, check_scan, check_trailers, hot_job, img_job,
                      mlp_job, run_jobs, scan_job)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cb_mode,io", [(0, "MAPPED"), (3, "MAPPED"), (3, "MAPPED_IN"), (3, "MAPPED_OUT")])
def test_mapped_io_all_copyless_types(cb_mode, io):
    s = S()
    jobs = ([blur_job(k) for k in range(4)] + [blur_job(50, W=17, H=3)] +
            [scan_job(100 + k, n=65536 - 999 * k) for k in range(4)] +
            [img_job(200 + k, dims=d) for k, d in enumerate([(300, 200), (129, 1), (1, 70), (640, 480)])] +
            [hot_job(300, R=37, C=100, K=13), hot_job(301, R=512, C=512, K=64)])
    slot = max(s.set_job_slot_bytes(j.type, s.dims4(*j.dims)) for j in jobs)
    st = run_jobs(jobs, num_streams=3, num_workers=2, ring_depth=2, slot_bytes=slot,
                  io_mode=getattr(s, "SET_IO_" + io), cb_mode=cb_mode)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        {1: check_blur, 2: check_scan, 3: check_img, 5: check_hot}[j.type](j)
    check_trailers(jobs)


def test_mapped_io_rejects_mlp_and_unmapped_buffers():
    s = S()
    slot = s.set_job_slot_bytes(s.SET_JOB_MLP_LN, s.dims4(16))
    ctx = s.create(s.default_config(num_streams=1, num_workers=1, slot_bytes=slot, io_mode=s.SET_IO_MAPPED))
    try:
        m = mlp_job(5, m=16)
        assert s.set_submit(ctx, ctypes.byref(m.desc), None) == s.SET_EINVAL
        # ordinary (pageable, unregistered) host memory: refused at submit, never touched by the GPU
        n = 4096
        xin = np.zeros(2 * n, np.float32)
        out = np.zeros(8 * n + 32, np.uint8)
        d = s.make_desc(s.SET_JOB_SAXPY_SCAN_MAX, (n,), xin.ctypes.data, out.ctypes.data, scalar=1.0)
        assert s.set_submit(ctx, ctypes.byref(d), None) == s.SET_EINVAL
        assert b"page-locked" in s.set_last_error(ctx)
        # device memory: refused too (the completion path reads the trailer from `out` on the host)
        j = scan_job(6, n=n, device=True)
        assert s.set_submit(ctx, ctypes.byref(j.desc), None) == s.SET_EINVAL
        assert b"not device memory" in s.set_last_error(ctx)
    finally:
        s.set_destroy(ctx)


def test_mapped_io_refuses_batches_and_baselines():
    s = S()
    cfg = s.default_config(num_streams=1, num_workers=1, slot_bytes=1 << 20, io_mode=s.SET_IO_MAPPED, batch_max=4)
    ctx = ctypes.c_void_p()
    assert s.set_create_ex(ctypes.byref(cfg), ctypes.byref(ctx)) == s.SET_EINVAL
    ctx = s.create(s.default_config(num_streams=1, num_workers=1, slot_bytes=1 << 20, io_mode=s.SET_IO_MAPPED))
    try:
        j = scan_job(7, n=1000)
        arr = (s.set_job_desc * 1)(j.desc)
        st = s.set_stats_t()
        assert s.set_run_baseline(ctx, s.SET_BASE_BATCH_SYNC, arr, 1, ctypes.byref(st)) == s.SET_EINVAL
    finally:
        s.set_destroy(ctx)


def test_mapped_output_mlp():
    # outputs stored by the kernels into host memory; x still copied (it feeds TMA loads)
    from gpu_util import check_mlp
    s = S()
    jobs = [mlp_job(600 + k, m=m) for k, m in enumerate([1, 77, 128, 200, 256])]
    slot = s.set_job_slot_bytes(s.SET_JOB_MLP_LN, s.dims4(256))
    st = run_jobs(jobs, num_streams=2, num_workers=1, slot_bytes=slot, io_mode=s.SET_IO_MAPPED_OUT, cb_mode=3)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        check_mlp(j)
    check_trailers(jobs)
