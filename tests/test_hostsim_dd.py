"""Host protocol of the device-dispatch lanes (set_dd_*) on CPU threads (no GPU).

The simulated backend (tests/hostsim/sim_dd.cpp, test-only) runs each launched loop on a host
thread that follows the fetch kernel's protocol on the same ring / control / completion layout:
retire the previous job, poll the next entry for idle_us, run the job (a delay and its trailer),
count an exit when no entry comes.  Checked: every job completes exactly once with its own
trailer, lanes whose loop ended are relaunched, a full ring gives SET_EAGAIN, wrong trailers are
reported, destroy drains; the same under ThreadSanitizer and AddressSanitizer.
"""
import ctypes
import os
import subprocess
import threading
import time

import numpy as np
import pytest

import hostsim_util
import paper_2606_05495_gb300 as B  # ctypes structs only; calls below go to the simulation library

DD_ENV = ("SET_SIM_DD_DELAY_US", "SET_SIM_DD_BADTRAILER_EVERY")
N_SCAN = 4096


@pytest.fixture
def sim():
    for k in DD_ENV:
        os.environ.pop(k, None)
    lib = hostsim_util.load()
    P = ctypes.POINTER
    vp, u64 = ctypes.c_void_p, ctypes.c_uint64
    lib.set_dd_config_default.argtypes = [P(B.set_dd_config)]
    lib.set_dd_create.argtypes = [P(B.set_dd_config), P(vp)]
    lib.set_dd_submit.argtypes = [vp, P(B.set_job_desc), P(u64)]
    lib.set_dd_submit_many.argtypes = [vp, P(B.set_job_desc), ctypes.c_size_t, P(u64), P(ctypes.c_size_t)]
    lib.set_dd_wait_all.argtypes = [vp, ctypes.c_int64]
    lib.set_dd_stats.argtypes = [vp, P(B.set_stats_t), P(u64)]
    lib.set_dd_destroy.argtypes = [vp]
    lib.set_dd_last_error.argtypes = [vp]
    lib.set_dd_last_error.restype = ctypes.c_char_p
    yield lib
    for k in DD_ENV:
        os.environ.pop(k, None)


class Jobs:
    """n scan-job descriptors over host buffers (the simulation only writes each trailer)."""

    def __init__(self, n):
        self.n = n
        dims = B.dims4(N_SCAN)
        self.in_b, self.out_b = B.set_job_in_bytes(2, dims), B.set_job_out_bytes(2, dims)
        self.inp = np.zeros(self.in_b + 64, np.uint8)
        self.out = np.zeros((n, self.out_b + 64), np.uint8)
        self.status = (ctypes.c_int32 * n)(*([99] * n))
        self.descs = (B.set_job_desc * n)()
        for k in range(n):
            d = self.descs[k]
            d.type, d.dims, d.in_, d.in_bytes = 2, dims, self.inp.ctypes.data, self.in_b
            d.out, d.out_bytes = self.out[k].ctypes.data, self.out_b
            d.status = ctypes.cast(ctypes.addressof(self.status) + 4 * k, ctypes.POINTER(ctypes.c_int32))

    def trailer(self, k):
        t = self.out[k, self.out_b - 16:self.out_b]
        return int(t[:8].view(np.uint64)[0]), int(t[8:12].view(np.uint32)[0]), int(t[12:16].view(np.uint32)[0])


def create(sim, **kw):
    c = B.set_dd_config()
    sim.set_dd_config_default(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    dd = ctypes.c_void_p()
    assert sim.set_dd_create(ctypes.byref(c), ctypes.byref(dd)) == B.SET_OK, sim.set_dd_last_error(None)
    return dd


def stats(sim, dd):
    st, launches = B.set_stats_t(), ctypes.c_uint64()
    assert sim.set_dd_stats(dd, ctypes.byref(st), ctypes.byref(launches)) == B.SET_OK
    return st, launches.value


def test_every_job_completes_once_with_its_trailer(sim):
    jobs = Jobs(600)
    dd = create(sim, num_lanes=5, ring_depth=4)
    first = ctypes.c_uint64()
    assert sim.set_dd_submit_many(dd, jobs.descs, jobs.n, ctypes.byref(first), None) == B.SET_OK
    assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
    st, launches = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK
    assert st.submitted == st.completed == jobs.n and st.failed == 0 and st.canary_errors == 0
    lanes = set()
    for k in range(jobs.n):
        jid, lane, word = jobs.trailer(k)
        assert jid == first.value + k and word == B.SET_TRAILER_MAGIC << 16 and jobs.status[k] == B.SET_OK
        lanes.add(lane)
    assert lanes == set(range(5))  # the shortest-lane choice spreads the groups of jobs
    assert launches >= 5


def test_concurrent_submitters(sim):
    jobs = Jobs(800)
    dd = create(sim, num_lanes=4, ring_depth=2, idle_us=100)
    ids = [None] * jobs.n

    def worker(t):
        for k in range(t, jobs.n, 4):
            jid = ctypes.c_uint64()
            assert sim.set_dd_submit(dd, ctypes.byref(jobs.descs[k]), ctypes.byref(jid)) == B.SET_OK
            ids[k] = jid.value

    th = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
    st, _ = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK
    assert st.completed == jobs.n and st.failed == 0 and len(set(ids)) == jobs.n
    for k in range(jobs.n):
        assert jobs.trailer(k)[0] == ids[k]


def test_idle_loops_end_and_are_relaunched(sim):
    jobs = Jobs(60)
    dd = create(sim, num_lanes=3, ring_depth=8, idle_us=100)
    for wave in range(4):
        sub = ctypes.cast(ctypes.addressof(jobs.descs) + wave * 15 * ctypes.sizeof(B.set_job_desc),
                          ctypes.POINTER(B.set_job_desc))
        assert sim.set_dd_submit_many(dd, sub, 15, None, None) == B.SET_OK
        assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
        time.sleep(0.02)  # far beyond idle_us: every loop ends
    st, launches = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK
    # set_dd_submit_many sends groups of up to 8 consecutive jobs to one lane: 15 jobs reach two
    # lanes per wave, whose loops ended during the previous wave's idle time
    assert st.completed == 60 and launches >= 4 * 2


def test_full_ring_nonblocking_and_blocking(sim):
    os.environ["SET_SIM_DD_DELAY_US"] = "30000,30000"  # 30 ms per job: the ring stays full
    jobs = Jobs(3)
    dd = create(sim, num_lanes=1, ring_depth=1)
    assert sim.set_dd_submit(dd, ctypes.byref(jobs.descs[0]), None) == B.SET_OK
    jobs.descs[1].flags = B.SET_F_NONBLOCK
    assert sim.set_dd_submit(dd, ctypes.byref(jobs.descs[1]), None) == B.SET_EAGAIN
    assert sim.set_dd_submit(dd, ctypes.byref(jobs.descs[2]), None) == B.SET_OK  # waits for room
    assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
    st, _ = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK
    assert st.submitted == 2 and st.completed == 2 and st.mem_waits == 1


def test_wrong_trailers_are_reported(sim):
    os.environ["SET_SIM_DD_BADTRAILER_EVERY"] = "7"
    jobs = Jobs(140)
    dd = create(sim, num_lanes=2, ring_depth=4)
    assert sim.set_dd_submit_many(dd, jobs.descs, jobs.n, None, None) == B.SET_OK
    assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
    st, _ = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK
    assert st.completed == 140 and st.canary_errors == 20 and st.failed == 20
    assert sum(1 for k in range(jobs.n) if jobs.status[k] == B.SET_EDEVICE) == 20


def test_destroy_drains_jobs_in_flight(sim):
    jobs = Jobs(300)
    dd = create(sim, num_lanes=3, ring_depth=2)
    assert sim.set_dd_submit_many(dd, jobs.descs, jobs.n, None, None) == B.SET_OK
    assert sim.set_dd_destroy(dd) == B.SET_OK
    assert all(jobs.status[k] == B.SET_OK for k in range(jobs.n))


def test_refused_descriptors(sim):
    jobs = Jobs(1)
    dd = create(sim, num_lanes=1, scan_max_n=1024)
    assert sim.set_dd_submit(dd, ctypes.byref(jobs.descs[0]), None) == B.SET_EINVAL  # n > scan_max_n
    assert b"scan_max_n" in sim.set_dd_last_error(dd)
    d = B.set_job_desc()
    d.type = B.SET_JOB_HOTSPOT  # several launches per job: not a lane kind
    d.dims = B.dims4(8, 8, 2)
    assert sim.set_dd_submit(dd, ctypes.byref(d), None) == B.SET_EINVAL
    assert b"only" in sim.set_dd_last_error(dd)
    st, _ = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK and st.submitted == 0


@pytest.mark.parametrize("san", ["thread", "address"])
def test_sanitizer_stress(san):
    exe = hostsim_util.build_stress(san, "stress_dd")
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 exitcode=66", ASAN_OPTIONS="detect_leaks=1 exitcode=66")
    for k in DD_ENV:
        env.pop(k, None)
    # (jobs, lanes, ring, idle_us): the short idle limits make loops end and relaunch constantly
    for args in (("3000", "5", "4", "200"), ("3000", "2", "1", "50"), ("2000", "1", "1", "10")):
        r = subprocess.run([exe, *args], capture_output=True, text=True, env=env, timeout=600)
        assert r.returncode == 0, (args, r.stdout + r.stderr[-3000:])


def test_reset_stats_keeps_jobs_in_flight_counted(sim):
    sim.set_dd_reset_stats.argtypes = [ctypes.c_void_p]
    jobs = Jobs(200)
    dd = create(sim, num_lanes=2, ring_depth=4)
    half = ctypes.cast(ctypes.addressof(jobs.descs) + 100 * ctypes.sizeof(B.set_job_desc),
                       ctypes.POINTER(B.set_job_desc))
    assert sim.set_dd_submit_many(dd, jobs.descs, 100, None, None) == B.SET_OK
    assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
    assert sim.set_dd_reset_stats(dd) == B.SET_OK
    st, _ = stats(sim, dd)
    assert st.submitted == 0 and st.completed == 0 and st.p99_us == 0
    assert sim.set_dd_submit_many(dd, half, 100, None, None) == B.SET_OK
    assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
    st, _ = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK
    assert st.submitted == 100 and st.completed == 100 and st.jobs_per_s > 0 and st.p50_us > 0


def test_queued_scan_jobs_retire_in_batches(sim):
    # one lane, a deep ring and a slow simulated job: descriptors queue up behind the running one,
    # so the loop takes several at once (up to the batch size) and retires them together with one
    # jump of the done counter; every job still completes once with its own trailer
    os.environ["SET_SIM_DD_DELAY_US"] = "200,400"
    sim.set_sim_dd_batched_jobs.restype = ctypes.c_uint64
    before = sim.set_sim_dd_batched_jobs()
    jobs = Jobs(300)
    dd = create(sim, num_lanes=1, ring_depth=32)
    first = ctypes.c_uint64()
    assert sim.set_dd_submit_many(dd, jobs.descs, jobs.n, ctypes.byref(first), None) == B.SET_OK
    assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
    st, _ = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK
    assert st.completed == jobs.n and st.failed == 0 and st.canary_errors == 0
    for k in range(jobs.n):
        assert jobs.trailer(k)[0] == first.value + k and jobs.status[k] == B.SET_OK
    assert sim.set_sim_dd_batched_jobs() - before >= jobs.n // 2


def test_submit_many_stops_at_an_invalid_job(sim):
    # the jobs before the invalid one are published (in groups) and complete with consecutive ids;
    # n_done is the invalid job's index and nothing after it is submitted
    jobs = Jobs(20)
    jobs.descs[13].in_bytes += 4
    dd = create(sim, num_lanes=2, ring_depth=16)
    first, done = ctypes.c_uint64(), ctypes.c_size_t()
    assert sim.set_dd_submit_many(dd, jobs.descs, jobs.n, ctypes.byref(first), ctypes.byref(done)) == B.SET_EINVAL
    assert done.value == 13 and b"in_bytes" in sim.set_dd_last_error(dd)
    assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
    st, _ = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK
    assert st.submitted == st.completed == 13 and st.failed == 0
    for k in range(13):
        assert jobs.trailer(k)[0] == first.value + k and jobs.status[k] == B.SET_OK
    assert all(jobs.status[k] == 99 for k in range(13, 20))


def test_submit_many_nonblocking_publishes_what_fits(sim):
    os.environ["SET_SIM_DD_DELAY_US"] = "30000,30000"  # the first job holds the lane for 30 ms
    jobs = Jobs(10)
    for k in range(jobs.n):
        jobs.descs[k].flags = B.SET_F_NONBLOCK
    dd = create(sim, num_lanes=1, ring_depth=4)
    first, done = ctypes.c_uint64(), ctypes.c_size_t()
    assert sim.set_dd_submit_many(dd, jobs.descs, jobs.n, ctypes.byref(first), ctypes.byref(done)) == B.SET_EAGAIN
    assert done.value == 4
    assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
    st, _ = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK
    assert st.submitted == st.completed == 4 and st.failed == 0
    for k in range(4):
        assert jobs.trailer(k)[0] == first.value + k and jobs.status[k] == B.SET_OK


def test_queued_blur_jobs_retire_in_batches(sim):
    # as the scan case, with blur descriptors: runs of the same kind are taken together
    os.environ["SET_SIM_DD_DELAY_US"] = "200,400"
    sim.set_sim_dd_batched_jobs.restype = ctypes.c_uint64
    before = sim.set_sim_dd_batched_jobs()
    n = 160
    dims = B.dims4(64, 32)
    in_b, out_b = B.set_job_in_bytes(B.SET_JOB_BLUR_HIST, dims), B.set_job_out_bytes(B.SET_JOB_BLUR_HIST, dims)
    inp = np.zeros(in_b + 64, np.uint8)
    out = np.zeros((n, out_b + 64), np.uint8)
    status = (ctypes.c_int32 * n)(*([99] * n))
    descs = (B.set_job_desc * n)()
    for k in range(n):
        d = descs[k]
        d.type, d.dims, d.in_, d.in_bytes = B.SET_JOB_BLUR_HIST, dims, inp.ctypes.data, in_b
        d.out, d.out_bytes = out[k].ctypes.data, out_b
        d.status = ctypes.cast(ctypes.addressof(status) + 4 * k, ctypes.POINTER(ctypes.c_int32))
    dd = create(sim, num_lanes=1, ring_depth=32)
    first = ctypes.c_uint64()
    assert sim.set_dd_submit_many(dd, descs, n, ctypes.byref(first), None) == B.SET_OK
    assert sim.set_dd_wait_all(dd, 60_000_000) == B.SET_OK
    st, _ = stats(sim, dd)
    assert sim.set_dd_destroy(dd) == B.SET_OK
    assert st.completed == n and st.failed == 0 and st.canary_errors == 0
    for k in range(n):
        jid = int(out[k, out_b - 16:out_b - 8].view(np.uint64)[0])
        assert jid == first.value + k and status[k] == B.SET_OK
    assert sim.set_sim_dd_batched_jobs() - before >= n // 2


def test_range_cache_edges(sim):
    # the per-call memory of accepted device allocations: containment at both ends, no
    # wrap-around for a start past the end, eviction of the oldest range
    sim.set_sim_dd_range_cache_check.restype = ctypes.c_uint32
    assert sim.set_sim_dd_range_cache_check() == 0
