"""set_config.guards: guard bands around every job's in / out / scratch regions, armed before the
job and checked after its last stage kernel.  Every stage kernel must leave them intact (a bounds
check in place of compute-sanitizer), and a planted change must be reported."""
import pytest

from gpu_util import (S, blur_job, check_any, check_trailers, hot_job, img_job, mlp_job, run_jobs, scan_job)

pytestmark = pytest.mark.gpu


def _slot(jobs):
    s = S()
    return max(s.set_job_slot_bytes(j.type, s.dims4(*j.dims)) for j in jobs) + 8192


@pytest.mark.parametrize("img_fused", [1, 0])
def test_no_stage_kernel_writes_outside_its_regions(img_fused):
    jobs = ([blur_job(1, W=17, H=3), blur_job(2), blur_job(3, W=1, H=1)] +
            [scan_job(10 + k, n=n) for k, n in enumerate([1, 3, 4097, 65536, 100003])] +
            [img_job(20 + k, dims=d) for k, d in enumerate([(1, 1), (5, 3), (129, 257), (700, 33), (640, 480)])] +
            [mlp_job(30 + k, m=m) for k, m in enumerate([1, 77, 256])] +
            [hot_job(40, R=37, C=100, K=13), hot_job(41, R=1, C=1, K=1), hot_job(42, R=512, C=512, K=64)])
    st = run_jobs(jobs, num_streams=3, num_workers=2, ring_depth=2, slot_bytes=_slot(jobs), guards=1,
                  img_fused=img_fused, cb_mode=3)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        check_any(j)
    check_trailers(jobs)


def test_a_changed_band_is_reported():
    s = S()
    jobs = [scan_job(50 + k, n=5000) for k in range(4)] + [blur_job(60 + k) for k in range(2)]
    jobs[1].desc.flags = s.SET_F_TEST_GUARD
    jobs[4].desc.flags = s.SET_F_TEST_GUARD
    st = run_jobs(jobs, num_streams=1, num_workers=1, ring_depth=1, slot_bytes=_slot(jobs), guards=1)
    assert st["completed"] == 6 and st["failed"] == 2 and st["canary_errors"] == 0, st
    for k, j in enumerate(jobs):
        _, _, word = j.trailer()
        if k in (1, 4):
            assert j.status.value == s.SET_EDEVICE and word == (s.SET_TRAILER_MAGIC << 16) | s.SET_DEVERR_GUARD
        else:
            assert j.status.value == s.SET_OK
            check_any(j)
