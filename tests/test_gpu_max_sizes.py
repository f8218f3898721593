"""Largest jobs the ABI accepts, end to end through the executor against the oracle: scan
n = 2^26, blur 2048 x 65535, image 4096 x 4096, hotspot at its longest sides."""
import numpy as np
import pytest

from gpu_util import S, check_blur, check_hot, check_img, check_scan, check_trailers, hot_job, img_job, run_jobs
from gpu_util import Job, scan_job

pytestmark = pytest.mark.gpu


def _one(job, **cfg):
    s = S()
    slot = s.set_job_slot_bytes(job.type, s.dims4(*job.dims))
    st = run_jobs([job], timeout_s=300, num_streams=1, num_workers=1, ring_depth=1, slot_bytes=slot, cb_mode=3, **cfg)
    assert st["completed"] == 1 and st["failed"] == 0 and st["canary_errors"] == 0, st
    check_trailers([job])


def test_scan_largest_n():
    job = scan_job(3, n=1 << 26)  # 512 MiB in, 16384 tiles
    _one(job)
    check_scan(job)


def test_blur_largest_image():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (65535, 2048), dtype=np.uint8)
    job = Job(S().SET_JOB_BLUR_HIST, (2048, 65535), img)
    _one(job)
    check_blur(job)


@pytest.mark.parametrize("fused", [1, 0])
def test_image_largest_sides(fused):
    job = img_job(7, dims=(4096, 4096))
    _one(job, img_fused=fused)
    check_img(job)


@pytest.mark.parametrize("C,R,K", [(8192, 16, 64), (16, 8192, 64), (2048, 2048, 8)])
def test_hotspot_longest_sides(C, R, K):
    job = hot_job(11, R=R, C=C, K=K)
    _one(job)
    check_hot(job)
