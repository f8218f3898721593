"""Hotspot job (compact thermal RC grid, K explicit steps, a chain of 8 temporally blocked
kernels) against the fp64 oracle: every cell within 1e-5 relative."""
import ctypes

import numpy as np
import pytest

import datagen
from gpu_util import S, check_hot, check_trailers, hot_job, run_jobs

pytestmark = pytest.mark.gpu

# (C, R, K): single cells and lines, C not a multiple of 4 (4-byte staging), several 64 x 64
# tiles with ragged tails, K below the number of launches (launches of zero steps) and at its
# maximum of 64 (8 steps per launch, the full halo)
SMALL = [(1, 1, 1), (1, 37, 5), (37, 1, 9), (100, 37, 13), (64, 64, 64), (65, 130, 64), (128, 96, 17),
         (300, 200, 64), (256, 8, 3)]


@pytest.mark.parametrize("C,R,K", SMALL)
def test_hotspot_small_and_ragged(C, R, K):
    jobs = [hot_job(7000 + C + R + K, R=R, C=C, K=K)]
    slot = S().set_job_slot_bytes(S().SET_JOB_HOTSPOT, S().dims4(C, R, K))
    st = run_jobs(jobs, num_streams=1, num_workers=1, slot_bytes=slot)
    assert st["completed"] == 1 and st["failed"] == 0 and st["canary_errors"] == 0
    check_hot(jobs[0])
    check_trailers(jobs)


def test_hotspot_full_size_through_lanes_with_slot_reuse():
    # 512 x 512 cells, 64 steps: the workload size; 12 jobs on 3 lanes x 2 slots, so slots (and
    # the last launch's CTA counter) are reused
    jobs = [hot_job(k) for k in range(12)]
    slot = S().set_job_slot_bytes(S().SET_JOB_HOTSPOT, S().dims4(512, 512, 64))
    st = run_jobs(jobs, num_streams=3, num_workers=1, ring_depth=2, slot_bytes=slot, cb_mode=3)
    assert st["completed"] == 12 and st["failed"] == 0 and st["canary_errors"] == 0
    worst = max(check_hot(j) for j in jobs)
    assert worst < 1e-5
    check_trailers(jobs)


def test_hotspot_mixed_sizes_and_device_io():
    # HBM-resident inputs and outputs; sizes and step counts differ from job to job on one slot set
    dims = [(512, 512, 64), (100, 37, 13), (513, 255, 40), (64, 64, 1), (512, 512, 64)]
    jobs = [hot_job(9000 + k, R=R, C=C, K=K, device=True) for k, (C, R, K) in enumerate(dims)]
    slot = max(S().set_job_slot_bytes(S().SET_JOB_HOTSPOT, S().dims4(*d)) for d in dims)
    st = run_jobs(jobs, num_streams=2, num_workers=1, ring_depth=1, slot_bytes=slot, io_mode=S().SET_IO_DEVICE)
    assert st["completed"] == len(jobs) and st["failed"] == 0
    for j in jobs:
        check_hot(j)
    check_trailers(jobs, io_host=False)


def test_hotspot_stage_order_stamps():
    # the 8 launches form a chain: each starts after its predecessor's last CTA has left
    jobs = [hot_job(9500 + k, R=200, C=160, K=64) for k in range(6)]
    slot = S().set_job_slot_bytes(S().SET_JOB_HOTSPOT, S().dims4(160, 200, 64))
    st = run_jobs(jobs, num_streams=2, num_workers=1, slot_bytes=slot, stamps=1)
    assert st["completed"] == 6 and st["failed"] == 0 and st["order_errors"] == 0
    for j in jobs:
        check_hot(j)


def test_hotspot_rejects_bad_dims():
    s = S()
    for dims in [(16, 16, 0), (16, 16, 65), (0, 16, 4), (16, 8193, 4)]:
        assert s.set_job_in_bytes(s.SET_JOB_HOTSPOT, s.dims4(*dims)) == 0, dims
