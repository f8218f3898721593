"""Scheduler invariant: per-job stage order, checked with device-written sequence stamps.

Every stage kernel's first CTA takes an entry ticket and its last CTA an exit ticket from one
device counter; the completion path asserts that each kernel entered after every kernel it
depends on had exited (chains: gray -> gauss -> sobel; DAG: {LayerNorm, GEMM1} -> GEMM2)."""
import pytest

from gpu_util import S, blur_job, check_any, check_trailers, img_job, mlp_job, run_jobs, scan_job

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fused,batch_max", [(0, 1), (1, 1), (1, 8)])
def test_stage_order_stamps(fused, batch_max):
    jobs = []
    for k in range(36):
        jobs.append([blur_job(k), scan_job(k, n=50000 + k), img_job(k, dims=(300 + k, 200)), mlp_job(k, m=1 + 7 * k)][k % 4])
    st = run_jobs(jobs, num_streams=3, num_workers=1, ring_depth=2, slot_bytes=32 << 20, stamps=1, img_fused=fused,
                  batch_max=batch_max)
    assert st["completed"] == 36 and st["failed"] == 0 and st["order_errors"] == 0 and st["canary_errors"] == 0
    for j in jobs:
        check_any(j)
    check_trailers(jobs)
