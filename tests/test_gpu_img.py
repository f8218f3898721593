"""GPU parity of the image job (gray -> Gauss5 -> Sobel -> histogram), fused and per stage,
bit-exact against the CPU oracle, through the executor's C ABI."""
import pytest

import datagen
from gpu_util import S, check_img, check_trailers, img_job, run_jobs

pytestmark = pytest.mark.gpu

EDGE = [(1, 1), (1, 5), (5, 1), (2, 2), (3, 3), (7, 5), (16, 16), (17, 33), (128, 128), (129, 130), (513, 40),
        (2048, 37), (37, 700), (640, 480)]


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("W,H", EDGE)
def test_img_edge_sizes(W, H, fused):
    jobs = [img_job(k, dims=(W, H)) for k in range(2)]
    st = run_jobs(jobs, num_streams=2, num_workers=1, slot_bytes=16 << 20, img_fused=fused)
    assert st["failed"] == 0 and st["canary_errors"] == 0
    for j in jobs:
        check_img(j)
    check_trailers(jobs)


@pytest.mark.parametrize("fused", [1, 0])
def test_img_workload_distribution(fused):
    # the workload's own log-uniform sides (128..2048), 24 jobs on 4 lanes, slots reused
    jobs = [img_job(j) for j in range(24)]
    slot = max(S().set_job_slot_bytes(3, S().dims4(*j.dims)) for j in jobs)
    st = run_jobs(jobs, num_streams=4, num_workers=2, slot_bytes=slot, img_fused=fused)
    assert st["completed"] == 24 and st["failed"] == 0
    for j in jobs:
        check_img(j)
    check_trailers(jobs)


def test_img_largest_and_thin():
    jobs = [img_job(0, dims=(4096, 64)), img_job(1, dims=(64, 4096)), img_job(2, dims=(2048, 2048))]
    slot = max(S().set_job_slot_bytes(3, S().dims4(*j.dims)) for j in jobs)
    st = run_jobs(jobs, num_streams=2, num_workers=2, slot_bytes=slot)
    assert st["failed"] == 0
    for j in jobs:
        check_img(j)


def test_img_and_scan_and_blur_share_slots():
    from gpu_util import blur_job, check_blur, check_scan, scan_job
    jobs = []
    for k in range(30):
        jobs.append([img_job(k, dims=(100 + 13 * k, 90 + 7 * k)), scan_job(k, n=30000 + 999 * k), blur_job(k)][k % 3])
    st = run_jobs(jobs, num_streams=3, num_workers=2, slot_bytes=4 << 20)
    assert st["failed"] == 0
    for j in jobs:
        {3: check_img, 2: check_scan, 1: check_blur}[j.type](j)
    check_trailers(jobs)


@pytest.mark.parametrize("per_stage", [False, True])
def test_direct_launch_fused_and_per_stage(per_stage):
    import ctypes
    from gpu_util import torch
    s, t = S(), torch()
    dims = [(700, 33), (129, 257), (1, 1), (640, 480)]
    jobs = [img_job(300 + k, dims=d, device=True) for k, d in enumerate(dims)]
    scratch = t.zeros(max(s.set_job_scratch_bytes(3, s.dims4(*j.dims)) for j in jobs), dtype=t.uint8, device="cuda")
    stream = t.cuda.current_stream().cuda_stream
    for k, j in enumerate(jobs):
        if per_stage:
            j.desc.flags |= s.SET_F_PER_STAGE
        st = s.set_launch_job(ctypes.byref(j.desc), j.hin.data_ptr(), j.hout.data_ptr(), scratch.data_ptr(), 2000 + k, 0,
                              stream)
        assert st == 0
        t.cuda.synchronize()
        check_img(j)
        assert j.trailer()[0] == 2000 + k
