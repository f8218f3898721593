"""GPU parity of the device-dispatch lanes (set_dd_*): jobs fetched and run by looping lane graphs."""
import ctypes
import time

import numpy as np
import pytest

from gpu_util import S, blur_job, check_blur, check_scan, scan_job

pytestmark = pytest.mark.gpu


def run_dd(jobs, timeout_s=120, **cfg):
    """Submits every job through set_dd_submit_many, waits, destroys; returns (stats, launches)."""
    s = S()
    dd = s.dd_create(s.dd_default_config(**cfg))
    try:
        arr = (s.set_job_desc * len(jobs))(*[j.desc for j in jobs])
        first = ctypes.c_uint64()
        s.dd_check(s.set_dd_submit_many(dd, arr, len(jobs), ctypes.byref(first), None), "set_dd_submit_many", dd)
        s.dd_check(s.set_dd_wait_all(dd, int(timeout_s * 1e6)), "set_dd_wait_all", dd)
        for k, j in enumerate(jobs):
            j.id = first.value + k
        st, launches = s.set_stats_t(), ctypes.c_uint64()
        s.dd_check(s.set_dd_stats(dd, ctypes.byref(st), ctypes.byref(launches)), "set_dd_stats", dd)
        return st.as_dict(), launches.value
    finally:
        assert s.set_dd_destroy(dd) == s.SET_OK


def check_dd_trailers(jobs, lanes):
    s = S()
    for j in jobs:
        jid, gen, word = j.trailer()
        assert jid == j.id, (jid, j.id)
        assert gen < lanes, gen  # slot_gen carries the lane index
        assert word == (s.SET_TRAILER_MAGIC << 16), hex(word)
        assert j.status.value == s.SET_OK, j.status.value


def test_single_jobs_one_lane():
    jobs = [scan_job(1, n=65536, device=True), blur_job(2, device=True)]
    st, launches = run_dd(jobs, num_lanes=1)
    assert st["completed"] == 2 and st["failed"] == 0 and st["canary_errors"] == 0, st
    assert launches >= 1
    check_scan(jobs[0])
    check_blur(jobs[1])
    check_dd_trailers(jobs, 1)


def test_scan_jobs_hbm_resident_16_lanes():
    jobs = [scan_job(k, device=True) for k in range(512)]
    st, launches = run_dd(jobs, num_lanes=16)
    assert st["completed"] == 512 and st["failed"] == 0 and st["canary_errors"] == 0, st
    assert launches >= 1
    for j in jobs:
        check_scan(j)
    check_dd_trailers(jobs, 16)


def test_blur_jobs_hbm_resident():
    jobs = [blur_job(k, device=True) for k in range(64)]
    st, _ = run_dd(jobs, num_lanes=2)
    assert st["completed"] == 64 and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        check_blur(j)
    check_dd_trailers(jobs, 2)


def test_mixed_kinds_and_ragged_sizes_share_lanes():
    # one lane graph runs all three kinds (SWITCH) and sizes below its fixed launch shape (spare
    # scan blocks leave at once; the blur node's shared memory covers the widest image; the image
    # node's fixed grid pulls the work items of any image size from the lane's ticket)
    from gpu_util import check_img, img_job
    jobs = [img_job(500 + k, dims=d, device=True) for k, d in enumerate([(1, 1), (5, 3), (129, 257), (640, 480),
                                                                          (2048, 33), (33, 2048)])]
    for k, n in enumerate([1, 2, 5, 4095, 4096, 4097, 30001, 65535, 65536, 7, 100, 8192]):
        jobs.append(scan_job(300 + k, n=n, device=True))
    for k, (W, H) in enumerate([(1, 1), (1, 9), (9, 1), (16, 16), (17, 3), (255, 257), (256, 1000), (33, 7)]):
        jobs.append(blur_job(400 + k, W=W, H=H, device=True))
    order = np.random.default_rng(5).permutation(len(jobs))
    jobs = [jobs[i] for i in order]
    st, _ = run_dd(jobs, num_lanes=3, ring_depth=4)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        {1: check_blur, 2: check_scan, 3: check_img}[j.type](j)
    check_dd_trailers(jobs, 3)


def test_host_buffers_are_refused():
    # page-locked host in/out are refused at submit (nothing runs on the GPU for them)
    s = S()
    dd = s.dd_create(s.dd_default_config(num_lanes=1))
    try:
        for j in (scan_job(600, n=4096), blur_job(601, W=32, H=32)):
            assert s.set_dd_submit(dd, ctypes.byref(j.desc), None) == s.SET_EINVAL
            assert b"device memory" in s.set_dd_last_error(dd)
        st = s.set_stats_t()
        s.dd_check(s.set_dd_stats(dd, ctypes.byref(st), None), "stats", dd)
        assert st.submitted == 0
    finally:
        assert s.set_dd_destroy(dd) == s.SET_OK


def test_unaligned_device_buffers_are_refused():
    s, t = S(), __import__("torch")
    dd = s.dd_create(s.dd_default_config(num_lanes=1))
    try:
        n = 1000
        buf_in = t.zeros(8 * n + 64, dtype=t.uint8, device="cuda")
        buf_out = t.zeros(s.set_job_out_bytes(2, s.dims4(n)) + 64, dtype=t.uint8, device="cuda")
        d = s.make_desc(s.SET_JOB_SAXPY_SCAN_MAX, (n,), buf_in.data_ptr() + 4, buf_out.data_ptr())
        assert s.set_dd_submit(dd, ctypes.byref(d), None) == s.SET_EINVAL
        d = s.make_desc(s.SET_JOB_SAXPY_SCAN_MAX, (n,), buf_in.data_ptr(), buf_out.data_ptr() + 8)
        assert s.set_dd_submit(dd, ctypes.byref(d), None) == s.SET_EINVAL
    finally:
        assert s.set_dd_destroy(dd) == s.SET_OK


def test_idle_lanes_end_their_loop_and_are_relaunched():
    s = S()
    dd = s.dd_create(s.dd_default_config(num_lanes=2, idle_us=200))
    try:
        jobs = []
        launches = ctypes.c_uint64()
        st = s.set_stats_t()
        for wave in range(3):
            # 12 jobs: set_dd_submit_many sends a group of 8 to one lane and the other 4 to the other
            batch = [scan_job(800 + 20 * wave + k, n=10000 + k, device=True) for k in range(12)]
            arr = (s.set_job_desc * len(batch))(*[j.desc for j in batch])
            first = ctypes.c_uint64()
            s.dd_check(s.set_dd_submit_many(dd, arr, len(batch), ctypes.byref(first), None), "submit", dd)
            s.dd_check(s.set_dd_wait_all(dd, 60_000_000), "wait", dd)
            for k, j in enumerate(batch):
                j.id = first.value + k
            jobs += batch
            time.sleep(0.05)  # far beyond idle_us: both loops end
        s.dd_check(s.set_dd_stats(dd, ctypes.byref(st), ctypes.byref(launches)), "stats", dd)
        assert st.completed == 36 and st.failed == 0
        assert launches.value >= 6, launches.value  # each wave relaunched both lanes
    finally:
        assert s.set_dd_destroy(dd) == s.SET_OK
    for j in jobs:
        check_scan(j)
    check_dd_trailers(jobs, 2)


def test_bounded_device_wait_reports_and_lane_continues():
    s = S()
    jobs = [scan_job(900 + k, n=65536, device=True) for k in range(5)]
    jobs[2].desc.flags = s.SET_F_TEST_STALL
    st, _ = run_dd(jobs, num_lanes=1)
    assert st["completed"] == 5 and st["failed"] == 1 and st["canary_errors"] == 0, st
    assert jobs[2].status.value == s.SET_EDEVICE
    _, _, word = jobs[2].trailer()
    assert word == (s.SET_TRAILER_MAGIC << 16) | s.SET_DEVERR_WAIT, hex(word)
    for k in (0, 1, 3, 4):
        assert jobs[k].status.value == s.SET_OK
        check_scan(jobs[k])


def test_full_ring_nonblocking_submit_returns_eagain():
    s = S()
    dd = s.dd_create(s.dd_default_config(num_lanes=1, ring_depth=1))
    try:
        slow = scan_job(950, n=65536, device=True)
        slow.desc.flags = s.SET_F_TEST_STALL  # holds the lane's only entry for >= 0.1 s
        s.dd_check(s.set_dd_submit(dd, ctypes.byref(slow.desc), None), "submit", dd)
        nb = scan_job(951, n=4096, device=True)
        nb.desc.flags = s.SET_F_NONBLOCK
        assert s.set_dd_submit(dd, ctypes.byref(nb.desc), None) == s.SET_EAGAIN
        nb.desc.flags = 0
        jid = ctypes.c_uint64()
        s.dd_check(s.set_dd_submit(dd, ctypes.byref(nb.desc), ctypes.byref(jid)), "blocking submit", dd)
        nb.id = jid.value
        s.dd_check(s.set_dd_wait_all(dd, 60_000_000), "wait", dd)
        st = s.set_stats_t()
        s.dd_check(s.set_dd_stats(dd, ctypes.byref(st), None), "stats", dd)
        assert st.mem_waits >= 1 and st.completed == 2 and st.failed == 1
    finally:
        assert s.set_dd_destroy(dd) == s.SET_OK
    check_scan(nb)
    check_dd_trailers([nb], 1)


def test_rejects_what_a_lane_cannot_run():
    s, t = S(), __import__("torch")
    from gpu_util import hot_job
    dd = s.dd_create(s.dd_default_config(num_lanes=1, scan_max_n=8192, blur_max_w=64))
    try:
        big = scan_job(960, n=8193, device=True)
        wide = blur_job(961, W=65, H=4, device=True)
        hot = hot_job(962, R=16, C=16, K=2, device=True)  # several launches per job: not a lane kind
        for j in (big, wide, hot):
            assert s.set_dd_submit(dd, ctypes.byref(j.desc), None) == s.SET_EINVAL
        pageable_in = np.zeros(8 * 100, np.uint8)
        out = t.zeros(s.set_job_out_bytes(2, s.dims4(100)), dtype=t.uint8, device="cuda")
        d = s.make_desc(s.SET_JOB_SAXPY_SCAN_MAX, (100,), pageable_in.ctypes.data, out.data_ptr())
        assert s.set_dd_submit(dd, ctypes.byref(d), None) == s.SET_EINVAL
        assert b"device memory" in s.set_dd_last_error(dd)
        st = s.set_stats_t()
        s.dd_check(s.set_dd_stats(dd, ctypes.byref(st), None), "stats", dd)
        assert st.submitted == 0
    finally:
        assert s.set_dd_destroy(dd) == s.SET_OK


def test_destroy_with_jobs_in_flight_completes_them():
    s = S()
    jobs = [scan_job(1000 + k, n=30000 + 11 * k, device=True) for k in range(200)]
    dd = s.dd_create(s.dd_default_config(num_lanes=4, ring_depth=8))
    arr = (s.set_job_desc * len(jobs))(*[j.desc for j in jobs])
    first = ctypes.c_uint64()
    try:
        s.dd_check(s.set_dd_submit_many(dd, arr, len(jobs), ctypes.byref(first), None), "submit", dd)
    finally:
        assert s.set_dd_destroy(dd) == s.SET_OK
    for k, j in enumerate(jobs):
        j.id = first.value + k
        check_scan(j)
    check_dd_trailers(jobs, 4)


def test_concurrent_submitters():
    # four host threads submit interleaved shares at once (lane rings and their mutexes shared)
    import threading
    s = S()
    jobs = [scan_job(1100 + k, n=16384 + 5 * k, device=True) for k in range(160)] + \
           [blur_job(1300 + k, device=True) for k in range(32)]
    dd = s.dd_create(s.dd_default_config(num_lanes=6, ring_depth=8))
    ids = [None] * len(jobs)
    errs = []

    def worker(t):
        try:
            for k in range(t, len(jobs), 4):
                jid = ctypes.c_uint64()
                st = s.set_dd_submit(dd, ctypes.byref(jobs[k].desc), ctypes.byref(jid))
                if st != s.SET_OK:
                    errs.append((k, st))
                ids[k] = jid.value
        except Exception as e:  # pragma: no cover - surfaced below
            errs.append(e)

    try:
        threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert not errs, errs
        s.dd_check(s.set_dd_wait_all(dd, 120_000_000), "wait", dd)
        st = s.set_stats_t()
        s.dd_check(s.set_dd_stats(dd, ctypes.byref(st), None), "stats", dd)
        assert st.completed == len(jobs) and st.failed == 0 and st.canary_errors == 0
    finally:
        assert s.set_dd_destroy(dd) == s.SET_OK
    assert len(set(ids)) == len(jobs)
    for j, jid in zip(jobs, ids):
        j.id = jid
        (check_blur if j.type == s.SET_JOB_BLUR_HIST else check_scan)(j)
    check_dd_trailers(jobs, 6)


def test_image_jobs_of_the_workload_sizes():
    # image jobs of the workload's log-uniform sizes (sides 128..2048) through 4 lanes
    from gpu_util import check_img, img_job
    jobs = [img_job(k, device=True) for k in range(24)]
    st, _ = run_dd(jobs, num_lanes=4, ring_depth=4)
    assert st["completed"] == 24 and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        check_img(j)
    check_dd_trailers(jobs, 4)


def test_queued_scan_jobs_batched_with_ragged_sizes_and_other_kinds():
    # one lane with a deep ring: scan descriptors queue behind the running iteration and the fetch
    # kernel takes up to kDdBatch consecutive ones at once (one launch of the scan node, one
    # scratch area per job); blur and image jobs in between end a batch
    from gpu_util import check_img, img_job
    sizes = [65536, 1, 4097, 30001, 65535, 5, 4096, 8192, 100, 65536, 12289]
    jobs = []
    for k in range(300):
        if k % 23 == 22:
            jobs.append(blur_job(2000 + k, W=255, H=31, device=True))
        elif k % 41 == 40:
            jobs.append(img_job(2000 + k, dims=(129, 65), device=True))
        else:
            jobs.append(scan_job(2000 + k, n=sizes[k % len(sizes)], device=True))
    st, _ = run_dd(jobs, num_lanes=1, ring_depth=64)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        {1: check_blur, 2: check_scan, 3: check_img}[j.type](j)
    check_dd_trailers(jobs, 1)


def test_bounded_wait_inside_a_batch_fails_only_its_job():
    # the stalled job shares a scan-node launch with the jobs queued beside it; only it reports
    # the bounded wait, the others (their own scratch areas) complete exactly
    s = S()
    jobs = [scan_job(2500 + k, n=65536, device=True) for k in range(12)]
    jobs[5].desc.flags = s.SET_F_TEST_STALL
    st, _ = run_dd(jobs, num_lanes=1, ring_depth=16)
    assert st["completed"] == 12 and st["failed"] == 1 and st["canary_errors"] == 0, st
    assert jobs[5].status.value == s.SET_EDEVICE
    for k in range(12):
        if k != 5:
            assert jobs[k].status.value == s.SET_OK
            check_scan(jobs[k])


def test_concurrent_submit_many_threads():
    # four host threads each submit a share with set_dd_submit_many (groups of up to 8 jobs to one
    # lane at a time, under the lanes' mutexes); ids are unique, every job's trailer carries its id
    import threading
    s = S()
    jobs = [scan_job(3000 + k, n=(4096, 65000, 777, 20000)[k % 4] + k, device=True) for k in range(256)]
    dd = s.dd_create(s.dd_default_config(num_lanes=5, ring_depth=16))
    errs = []

    def worker(t):
        share = jobs[t * 64:(t + 1) * 64]
        arr = (s.set_job_desc * len(share))(*[j.desc for j in share])
        done = ctypes.c_size_t()
        st = s.set_dd_submit_many(dd, arr, len(share), None, ctypes.byref(done))
        if st != s.SET_OK or done.value != len(share):
            errs.append((t, st, done.value))

    try:
        threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert not errs, errs
        s.dd_check(s.set_dd_wait_all(dd, 120_000_000), "wait", dd)
        st = s.set_stats_t()
        s.dd_check(s.set_dd_stats(dd, ctypes.byref(st), None), "stats", dd)
        assert st.completed == len(jobs) and st.failed == 0 and st.canary_errors == 0
    finally:
        assert s.set_dd_destroy(dd) == s.SET_OK
    for j in jobs:
        j.id = j.trailer()[0]
        check_scan(j)
    assert len({j.id for j in jobs}) == len(jobs)
    check_dd_trailers(jobs, 5)


def test_buffer_running_past_its_allocation_is_refused():
    # the driver reports the allocation that holds a buffer's start; a buffer whose extent runs
    # past its end is refused at submit (nothing is published).  The allocation is a caching-
    # allocator segment of its own, and the test first asks the driver for its range itself, so
    # that it submits only when the refusal is certain.
    t = __import__("torch")
    s = S()
    t.cuda.empty_cache()
    seg = 20 << 20
    buf = t.empty(seg, dtype=t.uint8, device="cuda")
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError:
        pytest.skip("driver library not loadable by name")
    base, size = ctypes.c_uint64(), ctypes.c_size_t()
    if cu.cuMemGetAddressRange_v2(ctypes.byref(base), ctypes.byref(size), ctypes.c_uint64(buf.data_ptr())) != 0:
        pytest.skip("the driver reports no allocation range here")
    end = base.value + size.value
    assert base.value <= buf.data_ptr() < end
    n = 1000
    out_bytes = s.set_job_out_bytes(s.SET_JOB_SAXPY_SCAN_MAX, s.dims4(n))
    good = scan_job(3500, n=n, device=True)
    past = (end - 4096) & ~15  # 16-byte aligned, fewer than out_bytes left before the end
    assert end - past < out_bytes
    d = s.make_desc(s.SET_JOB_SAXPY_SCAN_MAX, (n,), good.hin.data_ptr(), past)
    dd = s.dd_create(s.dd_default_config(num_lanes=1))
    try:
        assert s.set_dd_submit(dd, ctypes.byref(d), None) == s.SET_EINVAL
        assert b"inside one allocation" in s.set_dd_last_error(dd)
        st = s.set_stats_t()
        s.dd_check(s.set_dd_stats(dd, ctypes.byref(st), None), "stats", dd)
        assert st.submitted == 0
        # the same job with its own output is accepted and runs
        jid = ctypes.c_uint64()
        s.dd_check(s.set_dd_submit(dd, ctypes.byref(good.desc), ctypes.byref(jid)), "submit", dd)
        good.id = jid.value
        s.dd_check(s.set_dd_wait_all(dd, 60_000_000), "wait", dd)
    finally:
        assert s.set_dd_destroy(dd) == s.SET_OK
    del buf
    check_scan(good)
    check_dd_trailers([good], 1)


def test_queued_blur_jobs_batched_in_runs_with_ragged_sizes():
    # runs of blur jobs of ragged sizes (one 8-CTA cluster each in a batch), broken by scan runs
    # and image jobs: every batch holds one kind, results exact, trailers their own
    from gpu_util import check_img, img_job
    dims = [(256, 256), (1, 1), (17, 3), (255, 257), (64, 1000), (9, 1), (256, 31), (100, 100), (33, 7)]
    jobs = []
    for k in range(240):
        if k % 30 in (12, 13, 14):
            jobs.append(scan_job(4000 + k, n=(1, 4097, 65536)[k % 3], device=True))
        elif k % 53 == 52:
            jobs.append(img_job(4000 + k, dims=(97, 41), device=True))
        else:
            W, H = dims[k % len(dims)]
            jobs.append(blur_job(4000 + k, W=W, H=H, device=True))
    st, _ = run_dd(jobs, num_lanes=1, ring_depth=64)
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canary_errors"] == 0, st
    for j in jobs:
        {1: check_blur, 2: check_scan, 3: check_img}[j.type](j)
    check_dd_trailers(jobs, 1)
