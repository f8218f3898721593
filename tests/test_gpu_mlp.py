"""GPU parity of the MLP fork/join job (tcgen05 BF16 GEMMs + LayerNorm) against the fp64 oracle,
through the executor's C ABI."""
import pytest

from gpu_util import S, check_mlp, check_trailers, mlp_job, run_jobs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [1, 2, 7, 31, 64, 127, 128, 129, 200, 255, 256])
def test_mlp_rows(m):
    jobs = [mlp_job(k, m=m) for k in range(2)]
    slot = S().set_job_slot_bytes(4, S().dims4(m))
    st = run_jobs(jobs, num_streams=2, num_workers=1, slot_bytes=slot)
    assert st["failed"] == 0 and st["canary_errors"] == 0, (st, [(j.status.value, j.trailer()) for j in jobs])
    for j in jobs:
        check_mlp(j)
    check_trailers(jobs)


def test_mlp_workload_distribution_many_lanes():
    jobs = [mlp_job(j) for j in range(48)]  # m uniform on 1..256
    slot = S().set_job_slot_bytes(4, S().dims4(256))
    st = run_jobs(jobs, num_streams=6, num_workers=1, slot_bytes=slot)
    assert st["completed"] == 48 and st["failed"] == 0
    for j in jobs:
        check_mlp(j)
    check_trailers(jobs)
