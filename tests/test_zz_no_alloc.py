"""set_launch_scan_static: the scan launch for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (a plugin whose process owns all GPU memory through another
allocator, or a latency-critical path where an allocation would synchronise the device), so this
entry point keeps the scan's scratch in a static device array inside the library.  Its output
must match the regular entry point (set_launch_job with a caller-provided scratch buffer) within
the scan tolerance, on consecutive calls that reuse the array.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import SCAN_RTOL, S, scan_job, torch

pytestmark = pytest.mark.gpu


def _launch_both(k, n, stream):
    s, t = S(), torch()
    job = scan_job(k, n=n, device=True)
    out_static = t.zeros_like(job.hout)
    assert s.set_launch_scan_static(ctypes.byref(job.desc), job.hin.data_ptr(), out_static.data_ptr(), 500 + k, 3,
                                    stream) == s.SET_OK
    scratch = t.zeros(s.set_job_scratch_bytes(2, s.dims4(n)), dtype=t.uint8, device="cuda")
    assert s.set_launch_job(ctypes.byref(job.desc), job.hin.data_ptr(), job.hout.data_ptr(), scratch.data_ptr(),
                            500 + k, 3, stream) == s.SET_OK
    t.cuda.synchronize()
    return job.out(), out_static.cpu().numpy()


def test_static_scratch_matches_regular_entry_point_on_consecutive_calls():
    stream = torch().cuda.current_stream().cuda_stream
    for k, n in enumerate([65536, 100003, 65536]):
        ref, got = _launch_both(k, n, stream)
        fr, fg = ref[:8 * n + 16].view(np.float32), got[:8 * n + 16].view(np.float32)
        assert np.array_equal(fg[:n], fr[:n])  # z
        z = fr[:n].astype(np.float64)
        A = np.concatenate([[0.0], np.cumsum(np.abs(z))[:-1]])  # sum_{j<i} |z_j|
        assert np.all(np.abs(fg[n:2 * n].astype(np.float64) - fr[n:2 * n]) <= SCAN_RTOL * A)
        assert abs(float(fg[2 * n]) - float(fr[2 * n])) <= SCAN_RTOL * float(A.max())
        assert np.array_equal(got[-16:], ref[-16:])  # trailer: job id, slot generation, magic


def test_static_scratch_rejects_n_beyond_its_size():
    s, t = S(), torch()
    job = scan_job(0, n=64, device=True)
    job.desc.dims[0] = (1 << 24) + 1
    st = s.set_launch_scan_static(ctypes.byref(job.desc), job.hin.data_ptr(), job.hout.data_ptr(), 0, 0,
                                  t.cuda.current_stream().cuda_stream)
    assert st == s.SET_EINVAL
    assert b"16777216" in s.set_last_error(None)
