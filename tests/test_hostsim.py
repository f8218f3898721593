"""Host logic of the executor on CPU threads (no GPU): Algorithms 1-3 over a simulated device.

The simulated device (tests/hostsim/sim_device.cpp, test-only) runs each launch on its lane's
host thread after a random delay, writes only the job's trailer and calls the completion path
from one callback thread, like the CUDA driver's host-function thread.  Faults are injected on
the host: lost callbacks, stale slot generations, failing launches.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import hostsim_util
import paper_2606_05495_gb300 as B  # ctypes structs only; calls below go to the simulation library

SIM_ENV = ("SET_SIM_DELAY_US", "SET_SIM_DROP_EVERY", "SET_SIM_BADGEN_EVERY", "SET_SIM_FAIL_EVERY", "SET_SIM_SLOW_LANE")


@pytest.fixture
def sim():
    for k in SIM_ENV:
        os.environ.pop(k, None)
    lib = hostsim_util.load()
    c_void_p, c_int, c_int64, c_size_t, c_uint64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_uint64
    lib.set_create_ex.argtypes = [ctypes.POINTER(B.set_config), ctypes.POINTER(c_void_p)]
    lib.set_submit.argtypes = [c_void_p, ctypes.POINTER(B.set_job_desc), ctypes.POINTER(c_uint64)]
    lib.set_submit_many.argtypes = [c_void_p, ctypes.POINTER(B.set_job_desc), c_size_t, ctypes.POINTER(c_uint64),
                                    ctypes.POINTER(c_size_t)]
    lib.set_wait_all.argtypes = [c_void_p, c_int64]
    lib.set_stats.argtypes = [c_void_p, ctypes.POINTER(B.set_stats_t)]
    lib.set_destroy.argtypes = [c_void_p]
    lib.set_config_default.argtypes = [ctypes.POINTER(B.set_config)]
    lib.set_last_error.argtypes = [c_void_p]
    lib.set_last_error.restype = ctypes.c_char_p
    yield lib
    for k in SIM_ENV:
        os.environ.pop(k, None)


class Jobs:
    """n tiny blur (or image) jobs, 16x16, with host in/out buffers; the simulation writes only
    trailers."""

    def __init__(self, n, flags=0, type_=1):
        self.dims = B.dims4(16, 16)
        self.inb = np.zeros(3 * 256, np.uint8)
        ob = B.set_job_out_bytes(type_, self.dims)
        self.out = np.zeros((n, ob), np.uint8)
        self.status = (ctypes.c_int32 * n)(*([99] * n))
        self.descs = (B.set_job_desc * n)()
        for k in range(n):
            d = self.descs[k]
            d.type, d.flags, d.dims = type_, flags, self.dims
            d.in_, d.in_bytes = self.inb.ctypes.data, B.set_job_in_bytes(type_, self.dims)
            d.out, d.out_bytes = self.out[k].ctypes.data, ob
            d.status = ctypes.cast(ctypes.byref(self.status, 4 * k), ctypes.POINTER(ctypes.c_int32))

    def trailer_ids(self):
        return self.out[:, -16:-8].copy().view(np.uint64).ravel()


def create(lib, **kw):
    cfg = B.set_config()
    lib.set_config_default(ctypes.byref(cfg))
    cfg.slot_bytes = 1 << 16
    for k, v in kw.items():
        setattr(cfg, k, v)
    ctx = ctypes.c_void_p()
    assert lib.set_create_ex(ctypes.byref(cfg), ctypes.byref(ctx)) == 0, lib.set_last_error(None)
    return ctx


def stats(lib, ctx):
    st = B.set_stats_t()
    assert lib.set_stats(ctx, ctypes.byref(st)) == 0
    return st


def submit_all(lib, ctx, jobs, n):
    first, done = ctypes.c_uint64(), ctypes.c_size_t()
    rc = lib.set_submit_many(ctx, jobs.descs, n, ctypes.byref(first), ctypes.byref(done))
    return rc, first.value, done.value


def test_every_job_completes_exactly_once(sim):
    os.environ["SET_SIM_DELAY_US"] = "1,40"
    n = 3000
    jobs = Jobs(n)
    ctx = create(sim, num_streams=5, num_workers=3, ring_depth=2, queue_capacity=2)
    rc, first, done = submit_all(sim, ctx, jobs, n)
    assert rc == 0 and done == n
    assert sim.set_wait_all(ctx, 30_000_000) == 0
    st = stats(sim, ctx)
    sim.set_destroy(ctx)
    assert st.submitted == st.completed == n and st.failed == 0 and st.canary_errors == 0, st.as_dict()
    assert np.array_equal(np.sort(jobs.trailer_ids()), np.arange(first, first + n, dtype=np.uint64))
    assert all(s == 0 for s in jobs.status)
    assert st.p50_us <= st.p99_us <= st.max_us * 1.02 + 1
    assert st.mean_kernel_gap_us != st.mean_kernel_gap_us  # NaN: no device trace was taken


def test_idle_lanes_steal_from_a_lane_that_falls_behind(sim):
    # Algorithm 2: a slot whose lane queue is empty takes the next job of lane (w + k) mod b.
    # Lane 0 runs 40x slower, so the other lanes empty their queues while lane 0 still holds jobs.
    os.environ["SET_SIM_DELAY_US"] = "20,30"
    os.environ["SET_SIM_SLOW_LANE"] = "0,40"
    n = 400
    jobs = Jobs(n)
    ctx = create(sim, num_streams=4, num_workers=1, ring_depth=1, queue_capacity=1000)
    rc, first, done = submit_all(sim, ctx, jobs, n)
    assert rc == 0 and done == n
    assert sim.set_wait_all(ctx, 60_000_000) == 0
    st = stats(sim, ctx)
    sim.set_destroy(ctx)
    assert st.completed == n and st.failed == 0 and st.canary_errors == 0
    assert np.array_equal(np.sort(jobs.trailer_ids()), np.arange(first, first + n, dtype=np.uint64))
    assert st.steals > 0


def test_no_steals_without_stealing(sim):
    os.environ["SET_SIM_DELAY_US"] = "20,30"
    os.environ["SET_SIM_SLOW_LANE"] = "0,40"
    n = 200
    jobs = Jobs(n)
    ctx = create(sim, num_streams=4, num_workers=1, ring_depth=1, queue_capacity=1000, steal=0)
    rc, first, done = submit_all(sim, ctx, jobs, n)
    assert rc == 0 and done == n
    assert sim.set_wait_all(ctx, 60_000_000) == 0
    st = stats(sim, ctx)
    sim.set_destroy(ctx)
    assert st.completed == n and st.failed == 0 and st.steals == 0


@pytest.mark.parametrize("every,lanes,ring", [(2, 3, 2), (4, 2, 1), (8, 5, 3), (3, 1, 1)])
def test_completion_groups_never_strand_slots(sim, every, lanes, ring):
    os.environ["SET_SIM_DELAY_US"] = "1,30"
    n = 700
    jobs = Jobs(n)
    ctx = create(sim, num_streams=lanes, num_workers=1, ring_depth=ring, cb_every=every)
    rc, first, done = submit_all(sim, ctx, jobs, n)
    assert rc == 0 and done == n
    assert sim.set_wait_all(ctx, 30_000_000) == 0
    st = stats(sim, ctx)
    sim.set_destroy(ctx)
    assert st.completed == n and st.failed == 0 and st.canary_errors == 0
    assert np.array_equal(np.sort(jobs.trailer_ids()), np.arange(first, first + n, dtype=np.uint64))


@pytest.mark.parametrize("batch_max,every", [(4, 1), (8, 3), (64, 2)])
def test_batches_complete_every_job_once(sim, batch_max, every):
    os.environ["SET_SIM_DELAY_US"] = "5,60"
    n = 900
    jobs = Jobs(n, type_=3)
    ctx = create(sim, num_streams=3, num_workers=1, ring_depth=2, batch_max=batch_max, cb_every=every,
                 slot_bytes=1 << 20)
    rc, first, done = submit_all(sim, ctx, jobs, n)
    assert rc == 0 and done == n
    assert sim.set_wait_all(ctx, 30_000_000) == 0
    st = stats(sim, ctx)
    sim.set_destroy(ctx)
    assert st.completed == n and st.failed == 0 and st.canary_errors == 0
    assert np.array_equal(np.sort(jobs.trailer_ids()), np.arange(first, first + n, dtype=np.uint64))


def test_no_steal_mode_keeps_jobs_on_their_lane(sim):
    os.environ["SET_SIM_DELAY_US"] = "1,30"
    n = 800
    jobs = Jobs(n)
    ctx = create(sim, num_streams=4, num_workers=2, steal=0)
    assert submit_all(sim, ctx, jobs, n)[0] == 0
    assert sim.set_wait_all(ctx, 30_000_000) == 0
    st = stats(sim, ctx)
    sim.set_destroy(ctx)
    assert st.completed == n and st.steals == 0 and st.failed == 0


def test_nonblocking_submit_reports_full_queues(sim):
    os.environ["SET_SIM_DELAY_US"] = "20000,20000"
    n = 40
    jobs = Jobs(n, flags=B.SET_F_NONBLOCK)
    ctx = create(sim, num_streams=1, num_workers=1, ring_depth=1, queue_capacity=2)
    rcs = [sim.set_submit(ctx, ctypes.byref(jobs.descs[k]), None) for k in range(n)]
    assert B.SET_EAGAIN in rcs and rcs[0] == 0
    accepted = sum(1 for r in rcs if r == 0)
    assert sim.set_wait_all(ctx, 30_000_000) == 0
    st = stats(sim, ctx)
    sim.set_destroy(ctx)
    assert st.completed == accepted


def test_lost_callback_makes_wait_all_time_out(sim):
    os.environ["SET_SIM_DELAY_US"] = "1,5"
    os.environ["SET_SIM_DROP_EVERY"] = "7"
    n = 20
    jobs = Jobs(n)
    ctx = create(sim, num_streams=2, num_workers=2, drain_timeout_ms=200)
    assert submit_all(sim, ctx, jobs, n)[0] == 0
    assert sim.set_wait_all(ctx, 300_000) == B.SET_ETIMEDOUT
    st = stats(sim, ctx)
    assert st.completed < n
    sim.set_destroy(ctx)  # bounded drain: returns although slots never came back


def test_canary_flags_stale_slot_generation(sim):
    os.environ["SET_SIM_DELAY_US"] = "1,5"
    os.environ["SET_SIM_BADGEN_EVERY"] = "5"
    n = 100
    jobs = Jobs(n)
    ctx = create(sim, num_streams=2, num_workers=2)
    assert submit_all(sim, ctx, jobs, n)[0] == 0
    assert sim.set_wait_all(ctx, 30_000_000) == 0
    st = stats(sim, ctx)
    sim.set_destroy(ctx)
    assert st.canary_errors == 20 and st.failed == 20
    assert sum(1 for s in jobs.status if s == B.SET_EDEVICE) == 20


def test_launch_failure_is_sticky_and_drains(sim):
    os.environ["SET_SIM_DELAY_US"] = "1,5"
    os.environ["SET_SIM_FAIL_EVERY"] = "10"
    n = 60
    jobs = Jobs(n)
    ctx = create(sim, num_streams=2, num_workers=2)
    rc, _, done = submit_all(sim, ctx, jobs, n)
    assert rc in (0, B.SET_ECUDA)
    assert sim.set_wait_all(ctx, 30_000_000) == B.SET_ECUDA
    st = stats(sim, ctx)
    assert st.completed == done and st.failed >= 1
    assert sim.set_submit(ctx, ctypes.byref(jobs.descs[0]), None) == B.SET_ECUDA
    assert b"simulated" in sim.set_last_error(ctx)
    sim.set_destroy(ctx)


def test_invalid_descriptors(sim):
    ctx = create(sim, num_streams=1, num_workers=1, slot_bytes=1 << 16)
    jobs = Jobs(1)
    d = jobs.descs[0]
    d.in_bytes = 255
    assert sim.set_submit(ctx, ctypes.byref(d), None) == B.SET_EINVAL
    d.in_bytes = 256
    d.type = 9
    assert sim.set_submit(ctx, ctypes.byref(d), None) == B.SET_EINVAL
    d.type = 1
    d.dims = B.dims4(2048, 64)  # 128 KiB image does not fit a 64 KiB slot
    d.in_bytes = B.set_job_in_bytes(1, d.dims)
    d.out_bytes = B.set_job_out_bytes(1, d.dims)
    assert sim.set_submit(ctx, ctypes.byref(d), None) == B.SET_ENOMEM
    d.dims = B.dims4(0, 4)
    assert sim.set_submit(ctx, ctypes.byref(d), None) == B.SET_EINVAL
    assert sim.set_wait_all(ctx, 1_000_000) == 0
    sim.set_destroy(ctx)


@pytest.mark.parametrize("san", ["thread", "address"])
def test_sanitizer_stress(san):
    exe = hostsim_util.build_stress(san)
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 exitcode=66", ASAN_OPTIONS="detect_leaks=1 exitcode=66",
               SET_SIM_DELAY_US="0,20")
    for k in ("SET_SIM_DROP_EVERY", "SET_SIM_BADGEN_EVERY", "SET_SIM_FAIL_EVERY", "SET_SIM_SLOW_LANE"):
        env.pop(k, None)
    for every, bind in (("1", "0"), ("3", "0"), ("1", "1"), ("3", "1"), ("1", "2")):
        r = subprocess.run([exe, "6000", every, bind], capture_output=True, text=True, env=env, timeout=600)
        assert r.returncode == 0, (every, bind, r.stdout + r.stderr[-3000:])


@pytest.mark.parametrize("workers,every,bind,arena", [(1, 1, 1, 0), (3, 1, 1, 0), (2, 4, 1, 0), (2, 1, 2, 0),
                                                     (1, 1, 2, 1 << 22), (2, 2, 1, 1 << 22)])
def test_bind_at_submit_every_job_once(sim, workers, every, bind, arena):
    # UpdateGraphParams at submit: the submitter binds a free slot, dispatch only launches; jobs
    # that find no free slot are bound at dispatch as usual
    os.environ["SET_SIM_DELAY_US"] = "1,30"
    n = 2000
    jobs = Jobs(n)
    ctx = create(sim, num_streams=4, num_workers=workers, ring_depth=2, queue_capacity=4, cb_every=every,
                 bind_at_submit=bind, arena_bytes=arena)
    rc, first, done = submit_all(sim, ctx, jobs, n)
    assert rc == 0 and done == n
    assert sim.set_wait_all(ctx, 30_000_000) == 0
    st = stats(sim, ctx)
    sim.set_destroy(ctx)
    assert st.submitted == st.completed == n and st.failed == 0 and st.canary_errors == 0, st.as_dict()
    assert np.array_equal(np.sort(jobs.trailer_ids()), np.arange(first, first + n, dtype=np.uint64))
    assert all(s == 0 for s in jobs.status)


def test_bind_at_submit_refused_with_batches(sim):
    for kw in (dict(batch_max=4), dict(bind_at_submit=3)):
        cfg = B.set_config()
        sim.set_config_default(ctypes.byref(cfg))
        cfg.slot_bytes = 1 << 16
        cfg.bind_at_submit = 1
        for k, v in kw.items():
            setattr(cfg, k, v)
        ctx = ctypes.c_void_p()
        assert sim.set_create_ex(ctypes.byref(cfg), ctypes.byref(ctx)) == B.SET_EINVAL
