#!/usr/bin/env python
"""Benchmark of the SET executor on one GB300 (or N replicas under torchrun).

Workload (the headline configuration): 4096 scan jobs, each saxpy -> exclusive prefix sum ->
max|S| over n = 65536 fp32 elements (x, y uniform [-1, 1), per-job a uniform [-2, 2)), 512 KiB
copied in and 512 KiB + 32 B copied out per job, 8 lane streams with rings of 4 slots, four host
dispatch threads, work stealing, completion detected by a thread polling each lane's oldest event.  A step is one pass of all 4096 jobs through the executor (submit, dispatch, graph
launch, H2D copy, kernel, D2H copy, completion callback) until set_wait_all returns.

Printed JSON line:
  value        jobs/s with job inputs and outputs resident in HBM, read and written in place by
               the kernels (SET_IO_DEVICE_INPLACE), whole job over all ranks;
               value_device_copy_nodes: the same with device-to-device copy nodes (SET_IO_DEVICE)
  e2e          the same through the C ABI with pinned host buffers (SET_IO_HOST: H2D and D2H
               inside the timed region, moved over NVLink-C2C by the copy kernels of
               set_config.sm_copies); e2e_copy_engines: the same with the paper's memcpy nodes
  roofline     the dominant kernel (saxpy_scan_max) timed alone with CUDA events per launch over
               a > L2 working set, against the measured HBM copy bandwidth
  pipeline     the bound max(sum H2D / B_h2d, sum D2H / B_d2h, sum (H2D + D2H) / B_bidir,
               jobs x isolated kernel time) from copy rates measured here (copy kernels for e2e,
               copy engines for e2e_copy_engines and the baselines), and e2e / bound
  baselines    single-stream launch loop and the batch-synchronous fixed-stream graph executor
               on the same jobs (pinned host buffers)
  cpu_baseline the CPU oracle on the host cores over a bounded sample of the same jobs

--impl reference times the CPU oracle alone (this paper has no released code; the oracle is the
reference arm).  Inputs are larger than L2 (2 GiB per direction), so no flush is needed between
steps.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "jobs/s, mean kernel gap (us), p99 latency vs batch-sync CUDA-graph baseline"
UNIT = "jobs/s"
N_ELEM = 65536
JOB_IN = 8 * N_ELEM
JOB_OUT = 8 * N_ELEM + 32
# dram__bytes_read.sum + dram__bytes_write.sum per launch of saxpy_scan_max_kernel, mean of three
# launches of one ncu capture (profiles/saxpy_scan_max_kernel__scan_n65536.md); reset to None
# whenever the kernel changes until it is captured again
SCAN_TRAFFIC_BYTES = 544427


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["set", "reference"], default="set")
    p.add_argument("--jobs", type=int, default=4096)
    p.add_argument("--streams", type=int, default=8, help="lanes (the scan configuration names 8 streams)")
    p.add_argument("--workers", type=int, default=4, help="host dispatch threads")
    p.add_argument("--ring", type=int, default=4)
    p.add_argument("--cb-mode", type=int, default=3, help="completion path (set_config.cb_mode); 3 = polled events")
    p.add_argument("--cb-every", type=int, default=1, help="jobs per completion callback and lane")
    p.add_argument("--no-baselines", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--kernel-only", type=int, default=0, metavar="LAUNCHES",
                   help="only launch the dominant kernel this many times (for ncu), then exit")
    p.add_argument("--lanes", type=int, default=64, help="device-dispatch arm (set_dd): lanes")
    p.add_argument("--no-dd-arm", dest="dd_arm", action="store_false",
                   help="leave out the device-dispatch arm (set_dd) of the scan line")
    p.add_argument("--workload", choices=["scan", "blur", "img", "mlp", "serve", "hot", "bind-study", "copy-rates",
                                          "dd-study"],
                   default="scan",
                   help="scan (default) is the headline line; the others measure the other workloads")
    p.add_argument("--per-stage", action="store_true", help="--kernel-only on images: the three-stage chain")
    p.add_argument("--copy-kernel", action="store_true",
                   help="--kernel-only on scan jobs: the sm_copies copy kernel (512 KiB host -> HBM) instead")
    p.add_argument("--clock-ms", type=float, default=25.0, help="clock sampling period in timed regions")
    p.add_argument("--rates", default="1000,2000,5000,10000,20000,35000,50000", help="serve: arrival rates (jobs/s)")
    return p.parse_args()


# ---------------------------------------------------------------- distributed plumbing

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            backend = "nccl" if _torch().cuda.is_available() else "gloo"
            if backend == "nccl":
                _torch().cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            if _torch().cuda.is_available():
                self.pg.barrier(device_ids=[self.local])
            else:
                self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        t = _torch()
        dev = "cuda" if t.cuda.is_available() else "cpu"
        x = t.tensor([v], dtype=t.float64, device=dev)
        self.pg.all_reduce(x, op=self.pg.ReduceOp.MAX)
        return float(x.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def _torch():
    import torch
    return torch


def shard(njobs: int, rank: int):
    """Job ids of one rank: every rank runs its own njobs jobs (weak scaling, no collective)."""
    return range(rank * njobs, (rank + 1) * njobs)


# ---------------------------------------------------------------- clocks

class Clocks:
    """SM clock and clock-event reasons, sampled only while a timed region runs (`with
    clocks.window():`).  NVML through ctypes, read-only queries every period_ms from a thread; if
    NVML cannot be opened, nvidia-smi every 200 ms over the whole span instead."""

    # clock-event reason bits of nvmlDeviceGetCurrentClocksEventReasons
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: float = 25.0):
        import threading
        self.index, self.rows, self.p, self.period = index, [], None, period_ms * 1e-3
        self._on, self._quit = threading.Event(), threading.Event()
        self.nvml, self.h = self._open_nvml(index)
        if self.nvml is not None:
            self.th = threading.Thread(target=self._loop, daemon=True)
            self.th.start()
            return
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    @staticmethod
    def _open_nvml(index):
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None, None
            h = ctypes.c_void_p()
            t = _torch()
            pr = t.cuda.get_device_properties(index)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
            if lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(h)) != 0 and \
                    lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
                return None, None
            return lib, h
        except (OSError, AttributeError, RuntimeError):
            return None, None

    def _sample(self):
        cur, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        lib, h = self.nvml, self.h
        if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(cur)) != 0:  # NVML_CLOCK_SM
            return
        lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
        f = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        if f(h, ctypes.byref(rs)) != 0:
            rs.value = 0
        self.rows.append((cur.value, mx.value, rs.value))

    def _loop(self):
        while not self._quit.is_set():
            if self._on.wait(0.05) and not self._quit.is_set():
                self._sample()
                time.sleep(self.period)

    def window(self):
        """Context manager: samples are taken only inside it."""
        import contextlib

        @contextlib.contextmanager
        def cm():
            self._on.set()
            try:
                yield
            finally:
                self._on.clear()
        return cm()

    def stop(self):
        if self.nvml is not None:
            self._quit.set()
            self._on.set()
            self.th.join()
            sm = [r[0] for r in self.rows]
            reasons = sorted({n for r in self.rows for b, n in self.REASONS.items() if r[2] & b})
            return {"sm_mhz": statistics.median(sm) if sm else None,
                    "sm_max_mhz": max(r[1] for r in self.rows) if self.rows else None,
                    "samples": len(self.rows), "source": f"nvml, {self.period * 1e3:g} ms, timed regions only", "reasons": reasons}
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(rows), "source": "nvidia-smi, 200 ms", "reasons": reasons}


# ---------------------------------------------------------------- the oracle (CPU baseline / reference)

def oracle_rate(job_ids, cpu_seconds: float, threads: int, max_distinct: int = 512):
    """CPU oracle jobs/s over a bounded sample: inputs are generated before timing (up to
    max_distinct distinct jobs, cycled), then jobs run on `threads` host threads (ctypes drops the
    GIL), about cpu_seconds of CPU work in all, cycling over the workload's jobs."""
    from concurrent.futures import ThreadPoolExecutor

    import datagen
    import oracle

    oracle.lib()
    inputs = [datagen.scan_job(j, n=N_ELEM) for j in job_ids[:max_distinct]]

    def one(k):
        a, xy = inputs[k % len(inputs)]
        oracle.job_saxpy_scan_max(a, xy[:N_ELEM], xy[N_ELEM:])

    t0 = time.perf_counter()
    one(0)
    per_job = time.perf_counter() - t0
    n = max(threads, int(cpu_seconds / max(per_job, 1e-6)))  # cycles over the workload's jobs
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(n)))
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def run_reference(args, d: Dist):
    if d.rank != 0:
        return
    threads = os.cpu_count() or 1
    ids = list(shard(args.jobs, 0))
    for _ in range(args.warmup):
        oracle_rate(ids[:threads], 0.2, threads)
    rates, total_jobs, total_t = [], 0, 0.0
    for _ in range(args.steps):
        r, n, dt = oracle_rate(ids, 4.0, threads)
        rates.append(r)
        total_jobs += n
        total_t += dt
    value = total_jobs / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded SplitMix64 inputs)",
        "config": {"workload": "scan jobs (saxpy -> exclusive scan -> max|S|), n=65536 fp32, 4096 jobs",
                   "jobs_per_step": args.jobs, "l2": "inputs > L2 (no flush needed)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{total_jobs} jobs over {args.steps} steps, each a bounded sample "
                                   f"(about 4 s of CPU work) of the 4096-job workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- the SET executor arm

class Workload:
    """Pinned host and HBM-resident copies of every job of this rank, plus descriptors."""

    def __init__(self, S, ids, device_index: int):
        import numpy as np

        import datagen
        t = _torch()
        self.ids = list(ids)
        nj = len(self.ids)
        self.h_in = t.empty(nj * JOB_IN, dtype=t.uint8, pin_memory=True)
        self.h_out = t.zeros(nj * JOB_OUT, dtype=t.uint8, pin_memory=True)
        hv = self.h_in.numpy().view(np.float32).reshape(nj, 2 * N_ELEM)
        self.scalars = []
        for k, j in enumerate(self.ids):
            a, _ = datagen.scan_job(j, n=N_ELEM, out=hv[k])
            self.scalars.append(a)
        dev = f"cuda:{device_index}"
        self.d_in = self.h_in.to(dev)
        self.d_out = t.zeros(nj * JOB_OUT, dtype=t.uint8, device=dev)
        self.descs_host = self._descs(S, self.h_in.data_ptr(), self.h_out.data_ptr())
        self.descs_dev = self._descs(S, self.d_in.data_ptr(), self.d_out.data_ptr())

    def _descs(self, S, in_base, out_base):
        arr = (S.set_job_desc * len(self.ids))()
        for k in range(len(self.ids)):
            arr[k] = S.make_desc(S.SET_JOB_SAXPY_SCAN_MAX, (N_ELEM,), in_base + k * JOB_IN, out_base + k * JOB_OUT,
                                 scalar=self.scalars[k])
        return arr


def _profiler_attached() -> bool:
    """True when a profiler has injected itself into this process (ncu, nsys): CUPTI activity
    tracing is then left to it."""
    return bool(os.environ.get("CUDA_INJECTION64_PATH"))


def run_step(S, ctx, descs, n):
    done = ctypes.c_size_t()
    S.check(S.set_submit_many(ctx, descs, n, None, ctypes.byref(done)), "set_submit_many", ctx)
    S.check(S.set_wait_all(ctx, 600_000_000), "set_wait_all", ctx)


def timed(S, ctx, descs, n, args, d: Dist, clocks: "Clocks | None" = None):
    """W warm-up steps, then K steps bracketed by CUDA events (a barrier and a synchronize on both
    sides); an event at every step boundary also gives the median step (stats["ms_step_median"])."""
    import contextlib
    t = _torch()
    for _ in range(args.warmup):
        run_step(S, ctx, descs, n)
    S.set_reset_stats(ctx)
    d.barrier()
    t.cuda.synchronize()
    ev = [t.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with clocks.window() if clocks is not None else contextlib.nullcontext():
        ev[0].record()
        for k in range(args.steps):
            run_step(S, ctx, descs, n)
            ev[k + 1].record()
        t.cuda.synchronize()
    d.barrier()
    ms = ev[0].elapsed_time(ev[-1]) / args.steps
    st = S.set_stats_t()
    S.set_stats(ctx, ctypes.byref(st))
    out = st.as_dict()
    out["ms_step_median"] = statistics.median(ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps))
    return d.max(ms), out


_SUBMIT_POOLS = {}


def run_step_dd(S, dd, descs, n, threads=1):
    """One step through set_dd: submit every job (from `threads` host threads, each a contiguous
    share of the descriptors), then wait for all."""
    if threads <= 1:
        done = ctypes.c_size_t()
        S.dd_check(S.set_dd_submit_many(dd, descs, n, None, ctypes.byref(done)), "set_dd_submit_many", dd)
    else:
        from concurrent.futures import ThreadPoolExecutor
        pool = _SUBMIT_POOLS.setdefault(threads, ThreadPoolExecutor(threads))
        sz = ctypes.sizeof(S.set_job_desc)

        def share(k):
            a, b = k * n // threads, (k + 1) * n // threads
            first = ctypes.cast(ctypes.addressof(descs) + a * sz, ctypes.POINTER(S.set_job_desc))
            return S.set_dd_submit_many(dd, first, b - a, None, None)

        for st in pool.map(share, range(threads)):
            S.dd_check(st, "set_dd_submit_many", dd)
    S.dd_check(S.set_dd_wait_all(dd, 600_000_000), "set_dd_wait_all", dd)


def timed_dd(S, dd, descs, n, args, d: Dist, threads=1):
    """timed() for the device-dispatch lanes (set_dd): W warm-up steps, then K steps between CUDA
    events with a synchronize on both sides; returns (ms per step, stats, lane graph launches)."""
    t = _torch()
    for _ in range(args.warmup):
        run_step_dd(S, dd, descs, n, threads)
    S.set_dd_reset_stats(dd)
    d.barrier()
    t.cuda.synchronize()
    e0, e1 = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        run_step_dd(S, dd, descs, n, threads)
    e1.record()
    t.cuda.synchronize()
    d.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    st, launches = S.set_stats_t(), ctypes.c_uint64()
    S.set_dd_stats(dd, ctypes.byref(st), ctypes.byref(launches))
    return d.max(ms), st.as_dict(), launches.value


def device_dispatch_arm(S, w: "Workload", lanes: int, dev_index: int, args, d: Dist, threads: int = 1):
    """The same HBM-resident scan jobs through set_dd (lane graphs that fetch and run jobs on the
    device).  No CUPTI trace: activity records of kernels launched by conditional graph nodes came
    back incomplete (12 of ~8,200 kernels in one run), so device-timeline gaps are not reported."""
    nj = len(w.ids)
    dd = S.dd_create(S.dd_default_config(num_lanes=lanes, device=dev_index))
    try:
        ms_d, st_d, launches = timed_dd(S, dd, w.descs_dev, nj, args, d, threads)
    finally:
        S.set_dd_destroy(dd)
    world = d.world
    alg = 16 * N_ELEM + 32  # per job: read x, y; write z, S; m + trailer
    gbs = nj * alg / (ms_d * 1e-3) / 1e9
    peak = _peaks().get("hbm_gbs", 6800.0)
    return {
        "value": world * nj / (ms_d * 1e-3), "unit": UNIT, "ms_per_step": ms_d, "lanes": lanes,
        "submit_threads": threads,
        "p50_us": st_d["p50_us"], "p99_us": st_d["p99_us"], "submit_us": st_d["mean_launch_us"],
        "graph_launches": launches, "failed": st_d["failed"], "canary_errors": st_d["canary_errors"],
        "hbm": {"achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak, "alg_bytes_per_job": alg,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
        "note": "set_dd: per lane one graph WHILE {fetch -> SWITCH {blur | scan | image}} looping on the device; "
                "the host writes one descriptor per job (no graph update, launch or callback per job); "
                "set_dd_submit_many groups up to 8 jobs per lane and a lane runs up to 8 queued scan jobs "
                "in one launch",
    }


def copy_rates(S, job_in: int, job_out: int, streams: int, reps: int = 2048, sm: bool = False):
    """Pinned copy rates (GB/s) at the job's own sizes, `streams` streams back to back, timed in C
    (set_copy_bandwidth): H2D alone, D2H alone, and H2D + D2H together (total bytes both ways); on
    the copy engines, or (sm) by the copy kernel of set_config.sm_copies."""
    out = {}
    base = 3 if sm else 0
    for name, nbytes, direction in (("h2d_gbs", job_in, 0), ("d2h_gbs", job_out, 1), ("bidir_total_gbs", job_in, 2)):
        g = ctypes.c_double()
        S.check(S.set_copy_bandwidth(nbytes, streams, reps, base + direction, ctypes.byref(g)), "set_copy_bandwidth")
        out[name] = g.value
    return out


def kernel_time(S, w: Workload, launches: int = 512):
    """Average duration (us) of the saxpy_scan_max kernel launched alone per job: CUDA events
    around each launch on the launching stream, inputs cycling over the > L2 resident set.  A
    sleep kernel holds the stream while all launches are enqueued, so the GPU never waits for the
    host between them and each event pair brackets device time only."""
    t = _torch()
    s = t.cuda.Stream()
    scratch = t.zeros(S.set_job_scratch_bytes(S.SET_JOB_SAXPY_SCAN_MAX, S.dims4(N_ELEM)), dtype=t.uint8,
                      device=w.d_in.device)
    nj = len(w.ids)
    evs = [(t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)) for _ in range(launches)]
    with t.cuda.stream(s):
        for k in range(32):
            d = w.descs_dev[k % nj]
            S.check(S.set_launch_job(ctypes.byref(d), d.in_, d.out, scratch.data_ptr(), k, 0, s.cuda_stream), "launch")
        s.synchronize()
        t.cuda._sleep(int(2e9 * 20e-6 * launches))  # ~20 us of host enqueue time per launch
        for k in range(launches):
            d = w.descs_dev[(k * 7) % nj]
            evs[k][0].record(s)
            S.set_launch_job(ctypes.byref(d), d.in_, d.out, scratch.data_ptr(), k, 0, s.cuda_stream)
            evs[k][1].record(s)
    s.synchronize()
    ts = [a.elapsed_time(b) * 1e3 for a, b in evs]
    return statistics.mean(ts), statistics.median(ts)


def kernel_only(S, w: Workload, launches: int, copy_kernel: bool = False):
    """Launches the dominant kernel alone `launches` times over the resident inputs (profiling);
    copy_kernel: the copy kernel of set_config.sm_copies moving one job's input (512 KiB) from
    page-locked host memory to HBM, over a 256 MiB working set (set_copy_bandwidth, 8 streams)."""
    t = _torch()
    if copy_kernel:
        g = ctypes.c_double()
        S.check(S.set_copy_bandwidth(JOB_IN, 8, launches, 3, ctypes.byref(g)), "set_copy_bandwidth")
        print(json.dumps({"kernel_only": "copy_kernel", "launches": 2 * launches, "h2d_gbs": g.value}), flush=True)
        return
    scratch = t.zeros(S.set_job_scratch_bytes(S.SET_JOB_SAXPY_SCAN_MAX, S.dims4(N_ELEM)), dtype=t.uint8,
                      device=w.d_in.device)
    s = t.cuda.current_stream().cuda_stream
    for k in range(launches):
        d = w.descs_dev[(k * 7) % len(w.ids)]
        S.check(S.set_launch_job(ctypes.byref(d), d.in_, d.out, scratch.data_ptr(), k, 0, s), "set_launch_job")
    t.cuda.synchronize()
    print(json.dumps({"kernel_only": "saxpy_scan_max_kernel", "launches": launches}), flush=True)


def run_set(args, d: Dist):
    t = _torch()
    import paper_2606_05495_gb300 as S

    dev_index = d.local if t.cuda.is_available() else 0
    t.cuda.set_device(dev_index)
    w = Workload(S, shard(args.jobs, d.rank), dev_index)
    if args.kernel_only:
        kernel_only(S, w, args.kernel_only, args.copy_kernel)
        return
    nj = len(w.ids)
    cfg = dict(num_streams=args.streams, num_workers=args.workers, slot_bytes=S.set_job_slot_bytes(
        S.SET_JOB_SAXPY_SCAN_MAX, S.dims4(N_ELEM)), ring_depth=args.ring, cb_mode=args.cb_mode,
        cb_every=args.cb_every, device=dev_index)

    # value: inputs and outputs resident in HBM, read and written in place by the kernels (the
    # job graph is its kernel alone); then the same with device-to-device copy nodes into the slot
    ctx_dev = S.create(S.default_config(io_mode=S.SET_IO_DEVICE_INPLACE, **cfg))
    clocks = Clocks(dev_index, args.clock_ms)
    ms_dev, st_dev = timed(S, ctx_dev, w.descs_dev, nj, args, d, clocks)
    S.set_destroy(ctx_dev)
    ctx_dc = S.create(S.default_config(io_mode=S.SET_IO_DEVICE, **cfg))
    ms_dc, st_dc = timed(S, ctx_dc, w.descs_dev, nj, args, d, clocks)
    S.set_destroy(ctx_dc)

    # e2e with Algorithm 3's host-function callbacks (cb_mode 0, one dispatch thread): one per job
    # as written, and one per group of 8 launches of a lane
    host_cb = {}
    for name, every in (("per_job", 1), ("groups_of_8", 8)):
        c1 = dict(cfg, cb_mode=0, cb_every=every, num_workers=1)
        ctx1 = S.create(S.default_config(io_mode=S.SET_IO_HOST, **c1))
        host_cb[name] = timed(S, ctx1, w.descs_host, nj, argparse.Namespace(warmup=2, steps=min(3, args.steps)), d)
        S.set_destroy(ctx1)

    # e2e: pinned host buffers, H2D/D2H inside the timed region, moved by the copy kernels of
    # set_config.sm_copies (the fastest way to move a 512 KiB job over NVLink-C2C, see copy_rates)
    ctx_sm = S.create(S.default_config(io_mode=S.SET_IO_HOST, sm_copies=1, **cfg))
    ms_host, st_host = timed(S, ctx_sm, w.descs_host, nj, args, d, clocks)
    # the same with the paper's copy nodes on the copy engines; the baselines run on this context
    ctx = S.create(S.default_config(io_mode=S.SET_IO_HOST, **cfg))
    ms_ce, st_ce = timed(S, ctx, w.descs_host, nj, args, d, clocks)
    clk = clocks.stop()
    baselines = {}
    if not args.no_baselines:
        for name, kind in (("single_stream_loop", S.SET_BASE_SYNC), ("batch_sync_graph", S.SET_BASE_BATCH_SYNC)):
            st = S.set_stats_t()
            S.check(S.set_run_baseline(ctx, kind, w.descs_host, nj, ctypes.byref(st)), name, ctx)  # warm-up
            runs = []
            for _ in range(max(1, min(args.steps, 3))):
                S.check(S.set_run_baseline(ctx, kind, w.descs_host, nj, ctypes.byref(st)), name, ctx)
                runs.append(st.as_dict())
            best = sorted(runs, key=lambda r: r["jobs_per_s"])[len(runs) // 2]
            baselines[name] = {"jobs_per_s": best["jobs_per_s"], "p50_us": best["p50_us"], "p99_us": best["p99_us"],
                               "streams": 1 if kind == S.SET_BASE_SYNC else args.streams}
    # one CUPTI-traced step of each (untimed): device-timeline gaps (Sec. 3.2, Eq. 2-4)
    traces = {}
    tr = S.set_trace_summary()
    if not _profiler_attached() and S.set_trace_start() == S.SET_OK:
        run_step(S, ctx_sm, w.descs_host, nj)
        S.set_trace_stop(ctypes.byref(tr))
        traces["set"] = tr.as_dict()
        if S.set_trace_start() == S.SET_OK:
            run_step(S, ctx, w.descs_host, nj)
            S.set_trace_stop(ctypes.byref(tr))
            traces["set_copy_engines"] = tr.as_dict()
        if not args.no_baselines and not _profiler_attached() and S.set_trace_start() == S.SET_OK:
            st = S.set_stats_t()
            S.set_run_baseline(ctx, S.SET_BASE_BATCH_SYNC, w.descs_host, nj, ctypes.byref(st))
            S.set_trace_stop(ctypes.byref(tr))
            traces["batch_sync_graph"] = tr.as_dict()
    S.set_destroy(ctx)
    S.set_destroy(ctx_sm)

    # UpdateGraphParams at submit (the submitting thread binds free slots) instead of at dispatch,
    # and the same pinned host buffers read and written by the kernels over the host link (no copy
    # nodes; SET_IO_MAPPED).  Skipped under a profiler: its launch list covers the headline arms.
    ms_bind = ms_map = None
    if not _profiler_attached():
        ctxb = S.create(S.default_config(io_mode=S.SET_IO_HOST, bind_at_submit=1, **cfg))
        ms_bind, st_bind = timed(S, ctxb, w.descs_host, nj, args, d)
        S.set_destroy(ctxb)
        ctxm = S.create(S.default_config(io_mode=S.SET_IO_MAPPED, **cfg))
        ms_map, st_map = timed(S, ctxm, w.descs_host, nj, args, d)
        S.set_destroy(ctxm)

    dd_arm = None
    if not _profiler_attached() and args.dd_arm:
        dd_arm = device_dispatch_arm(S, w, args.lanes, dev_index, args, d)

    k_mean_us, k_med_us = kernel_time(S, w)
    rates = copy_rates(S, JOB_IN, JOB_OUT, args.streams)
    # copy kernels gain from concurrency (unlike the engines): measured over as many streams as the
    # executor keeps jobs in flight (lanes x ring)
    rates_sm = copy_rates(S, JOB_IN, JOB_OUT, args.streams * args.ring, sm=True)
    # the link's ceiling for the e2e roofline: both directions at once with 64 MiB copies
    link = ctypes.c_double()
    S.check(S.set_copy_bandwidth(64 << 20, args.streams, 16, 2, ctypes.byref(link)), "set_copy_bandwidth")
    world = d.world
    value = world * nj / (ms_dev * 1e-3)
    e2e = world * nj / (ms_host * 1e-3)
    e2e_ce = world * nj / (ms_ce * 1e-3)

    alg_bytes = 16 * N_ELEM + 32  # read x, y; write z, S; m + trailer
    achieved = alg_bytes / (k_mean_us * 1e-6) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    t_h2d = nj * JOB_IN / (rates["h2d_gbs"] * 1e9)
    t_d2h = nj * JOB_OUT / (rates["d2h_gbs"] * 1e9)
    t_bi = nj * (JOB_IN + JOB_OUT) / (rates["bidir_total_gbs"] * 1e9)
    k_exec_us = traces.get("set", {}).get("top_kernel_mean_us") or k_mean_us
    sms = t.cuda.get_device_properties(dev_index).multi_processor_count
    t_sm = nj * k_exec_us * 1e-6 * 16 / sms  # 16 CTAs per job, one per SM: the share of SM time
    bound_s = max(t_h2d, t_d2h, t_bi, t_sm)
    bound_sm_s = max(nj * JOB_IN / (rates_sm["h2d_gbs"] * 1e9), nj * JOB_OUT / (rates_sm["d2h_gbs"] * 1e9),
                     nj * (JOB_IN + JOB_OUT) / (rates_sm["bidir_total_gbs"] * 1e9), t_sm)
    if d.rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_dev, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded SplitMix64 inputs, resident before timing)",
        "config": {"workload": "scan jobs (saxpy -> exclusive scan -> max|S|), n=65536 fp32, 4096 jobs per GPU",
                   "jobs_per_step": nj * world, "streams": args.streams, "workers": args.workers,
                   "ring_depth": args.ring, "cb_mode": args.cb_mode, "cb_every": args.cb_every, "steal": True,
                   "io": "HBM-resident in/out, read and written in place (SET_IO_DEVICE_INPLACE)",
                   "l2": "inputs 2 GiB > L2 per step (no flush needed)", "parallelism": f"replicas x{world}"},
        "value_device_copy_nodes": {"value": world * nj / (ms_dc * 1e-3), "unit": UNIT, "ms_per_step": ms_dc,
                                    "p99_us": st_dc["p99_us"], "mean_update_us": st_dc["mean_update_us"],
                                    "mean_launch_us": st_dc["mean_launch_us"],
                                    "note": "SET_IO_DEVICE: device-to-device copy nodes into the slot around "
                                            "the kernel"},
        "value_update_us": st_dev["mean_update_us"], "value_launch_us": st_dev["mean_launch_us"],
        "ms_per_step_median": st_dev["ms_step_median"],
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nj * JOB_IN, "d2h_bytes_per_step": nj * JOB_OUT,
                "ms_per_step": ms_host, "ms_per_step_median": st_host["ms_step_median"],
                "p50_us": st_host["p50_us"], "p99_us": st_host["p99_us"],
                "mean_update_us": st_host["mean_update_us"], "mean_launch_us": st_host["mean_launch_us"],
                "steals": st_host["steals"], "copies": "copy kernels over NVLink-C2C (set_config.sm_copies)",
                "note": "completion by polled events (cb_mode 3); H2D and D2H of every job by the copy kernels "
                        "of set_config.sm_copies in place of the graph's memcpy nodes"},
        "e2e_copy_engines": {
            "value": e2e_ce, "unit": UNIT, "h2d_bytes_per_step": nj * JOB_IN, "d2h_bytes_per_step": nj * JOB_OUT,
            "ms_per_step": ms_ce, "p50_us": st_ce["p50_us"], "p99_us": st_ce["p99_us"],
            "mean_update_us": st_ce["mean_update_us"], "mean_launch_us": st_ce["mean_launch_us"],
            "steals": st_ce["steals"],
            "host_callbacks": {k: {"value": world * nj / (v[0] * 1e-3), "p99_us": v[1]["p99_us"],
                                   "mean_launch_us": v[1]["mean_launch_us"]} for k, v in host_cb.items()},
            "note": "the paper's job graph: memcpy nodes on the copy engines, polled completion; host_callbacks: "
                    "cudaLaunchHostFunc on a callback stream (cb_mode 0), one dispatch thread; the baselines "
                    "run on this context"},
        "e2e_bind_at_submit": None if ms_bind is None else {
            "value": world * nj / (ms_bind * 1e-3), "unit": UNIT, "ms_per_step": ms_bind,
            "p99_us": st_bind["p99_us"], "mean_update_us": st_bind["mean_update_us"],
            "mean_launch_us": st_bind["mean_launch_us"],
            "note": "UpdateGraphParams on the submitting thread (set_config.bind_at_submit), copy engines"},
        "e2e_mapped": None if ms_map is None else {
            "value": world * nj / (ms_map * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nj * JOB_IN,
            "d2h_bytes_per_step": nj * JOB_OUT, "ms_per_step": ms_map, "p50_us": st_map["p50_us"],
            "p99_us": st_map["p99_us"],
            "note": "SET_IO_MAPPED: the same pinned host buffers, read and written by the kernels over "
                    "NVLink-C2C; the job graphs have no copy nodes"},
        "device_dispatch": dd_arm,
        "gpu_launches": args.steps * nj * 1,  # value's timed region: one kernel node per job
        "gpu_launches_e2e": args.steps * nj * 3,  # e2e's: copy-in kernel, stage kernel, copy-out kernel
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": SCAN_TRAFFIC_BYTES, "kernel": "saxpy_scan_max_kernel",
                     "kernel_us_mean": k_mean_us, "kernel_us_median": k_med_us,
                     "alg_bytes_per_launch": alg_bytes, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
        "roofline_e2e": {"bound": "c2c", "kernel": "copy_kernel (with saxpy_scan_max_kernel)",
                         "achieved": nj / (ms_host * 1e-3) * (JOB_IN + JOB_OUT) / 1e9, "peak": link.value,
                         "unit": "GB/s", "frac": nj / (ms_host * 1e-3) * (JOB_IN + JOB_OUT) / 1e9 / link.value,
                         "peak_source": "measured here: H2D + D2H together with 64 MiB copy-engine copies",
                         "note": "bytes moved over NVLink-C2C per second by the e2e arm (in + out per job)"},
        "pipeline": {"copy_kernel_rates_gbs": rates_sm, "copy_kernel_streams": args.streams * args.ring,
                     "bound_jobs_per_s": nj / bound_sm_s, "e2e_frac_of_bound": (nj / (ms_host * 1e-3)) / (nj / bound_sm_s),
                     "copy_engine_rates_gbs": rates, "copy_engine_bound_jobs_per_s": nj / bound_s,
                     "copy_engine_e2e_frac_of_bound": (nj / (ms_ce * 1e-3)) / (nj / bound_s),
                     "copy_engine_terms_ms": {"h2d": t_h2d * 1e3, "d2h": t_d2h * 1e3, "bidir": t_bi * 1e3,
                                              "sm": t_sm * 1e3}},
        "p99_us": st_host["p99_us"],
        "mean_kernel_gap_us": traces.get("set", {}).get("mean_kernel_gap_us"),
        "trace": {k: {f: v[f] for f in ("kernels", "memcpys", "span_us", "kernel_busy_us", "copy_busy_us",
                                        "idle_frac", "mean_kernel_gap_us", "max_kernel_gap_us", "top_kernel_mean_us")}
                  for k, v in traces.items()},
        "baselines": baselines, "clocks": clk,
    }
    # Eq. 4: t_schedule / T_measured = 1 - T_ideal / T_measured, T_ideal = the gap-free pipeline time
    t_ideal_ms = bound_s * 1e3  # copy-engine arms and baselines
    sched = {"set_e2e": 1 - bound_sm_s * 1e3 / ms_host, "set_copy_engines": 1 - t_ideal_ms / ms_ce}
    sched.update({f"set_host_callbacks_{k}": 1 - t_ideal_ms / v[0] for k, v in host_cb.items()})
    for k, v in baselines.items():
        sched[k] = 1 - v["jobs_per_s"] / (nj / bound_s)
    line["eq4_schedule_frac"] = sched
    if not args.no_cpu:
        threads = os.cpu_count() or 1
        ids = list(shard(args.jobs, 0))
        r, n, dt = oracle_rate(ids, 20.0, threads)  # about 20 s of CPU work over all threads
        r1, n1, dt1 = oracle_rate(ids, 3.0, 1)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{n} scan jobs cycling over the workload's {len(ids)} "
                                          f"({dt:.1f} s wall on {threads} threads)",
                                "single_thread": {"value": r1, "jobs": n1, "seconds": dt1}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- the other workloads

class JobSet:
    """Jobs of one kind with inputs / outputs in two pinned buffers (and device copies)."""

    def __init__(self, S, kind, ids, dims=None, device_copy=False):
        import numpy as np

        import datagen
        t = _torch()
        self.kind, self.ids = kind, list(ids)
        self.dims = []
        for k, j in enumerate(self.ids):
            if kind == 1:
                self.dims.append((256, 256))
            elif kind == 3:
                self.dims.append(dims[k] if dims else datagen.img_dims(j))
            elif kind == 5:
                self.dims.append(dims[k] if dims else (datagen.HOT_SIDE, datagen.HOT_SIDE, datagen.HOT_STEPS))
            else:
                self.dims.append((dims[k] if dims else datagen.mlp_rows(j),))
        ib = [S.set_job_in_bytes(kind, S.dims4(*d)) for d in self.dims]
        ob = [S.set_job_out_bytes(kind, S.dims4(*d)) for d in self.dims]
        self.in_off = np.concatenate([[0], np.cumsum([(b + 255) // 256 * 256 for b in ib])]).astype(np.int64)
        self.out_off = np.concatenate([[0], np.cumsum([(b + 255) // 256 * 256 for b in ob])]).astype(np.int64)
        self.h_in = t.empty(int(self.in_off[-1]), dtype=t.uint8, pin_memory=True)
        self.h_out = t.zeros(int(self.out_off[-1]), dtype=t.uint8, pin_memory=True)
        hv = self.h_in.numpy()
        for k, j in enumerate(self.ids):
            seg = hv[self.in_off[k]:self.in_off[k] + ib[k]]
            if kind == 1:
                datagen.blur_job(j, out=seg)
            elif kind == 3:
                datagen.img_job(j, out=seg, dims=self.dims[k])
            elif kind == 5:
                C, R, _ = self.dims[k]
                datagen.hot_job(j, R, C, out=seg.view(np.float32))
            else:
                datagen.mlp_job(j, out=seg.view(np.uint16), m=self.dims[k][0])
        self.shared = (None, None)
        if kind == 4:
            w1, w2 = datagen.mlp_weights()
            self.w = (t.from_numpy(w1.view(np.int16)).cuda(), t.from_numpy(w2.view(np.int16)).cuda())
            self.shared = (self.w[0].data_ptr(), self.w[1].data_ptr())
        self.bytes_in, self.bytes_out = sum(ib), sum(ob)
        self.descs = self._descs(S, self.h_in.data_ptr(), self.h_out.data_ptr())
        if device_copy:
            self.d_in = self.h_in.cuda()
            self.d_out = t.zeros_like(self.h_out, device="cuda")
            self.descs_dev = self._descs(S, self.d_in.data_ptr(), self.d_out.data_ptr())

    def _descs(self, S, ib, ob):
        arr = (S.set_job_desc * len(self.ids))()
        for k in range(len(self.ids)):
            arr[k] = S.make_desc(self.kind, self.dims[k], ib + int(self.in_off[k]), ob + int(self.out_off[k]),
                                 shared=self.shared)
        return arr

    def slot_bytes(self, S):
        return max(S.set_job_slot_bytes(self.kind, S.dims4(*d)) for d in self.dims)

    def rows(self):
        return sum(d[0] for d in self.dims)


def _rate(S, cfg, descs, n, args, d, clocks=None):
    """jobs/s of the SET executor over `steps` timed steps, with the stats of those steps."""
    ctx = S.create(S.default_config(**cfg))
    try:
        ms, st = timed(S, ctx, descs, n, args, d, clocks)
        return {"jobs_per_s": n / (ms * 1e-3), "ms_per_step": ms, "p50_us": st["p50_us"], "p99_us": st["p99_us"],
                "failed": st["failed"], "canary_errors": st["canary_errors"]}
    finally:
        S.set_destroy(ctx)


def _baseline(S, cfg, kind, descs, n):
    ctx = S.create(S.default_config(**cfg))
    try:
        st = S.set_stats_t()
        S.check(S.set_run_baseline(ctx, kind, descs, n, ctypes.byref(st)), "baseline", ctx)
        S.check(S.set_run_baseline(ctx, kind, descs, n, ctypes.byref(st)), "baseline", ctx)
        return {"jobs_per_s": st.jobs_per_s, "p50_us": st.p50_us, "p99_us": st.p99_us}
    finally:
        S.set_destroy(ctx)


TRACE_FIELDS = ("kernels", "memcpys", "span_us", "kernel_busy_us", "copy_busy_us", "idle_frac",
                "mean_kernel_gap_us", "max_kernel_gap_us", "top_kernel_mean_us")


def _traces(S, cfg, descs, n):
    """One CUPTI-traced (untimed) step of SET and one of the batch-synchronous baseline on the same
    jobs and slots: device-timeline gaps (Sec. 3.2, Eq. 2-4)."""
    out = {}
    if _profiler_attached():
        return out
    ctx = S.create(S.default_config(**cfg))
    try:
        run_step(S, ctx, descs, n)
        tr = S.set_trace_summary()
        if S.set_trace_start() == S.SET_OK:
            run_step(S, ctx, descs, n)
            S.set_trace_stop(ctypes.byref(tr))
            out["set"] = {f: getattr(tr, f) for f in TRACE_FIELDS}
        if S.set_trace_start() == S.SET_OK:
            st = S.set_stats_t()
            S.set_run_baseline(ctx, S.SET_BASE_BATCH_SYNC, descs, n, ctypes.byref(st))
            S.set_trace_stop(ctypes.byref(tr))
            out["batch_sync_graph"] = {f: getattr(tr, f) for f in TRACE_FIELDS}
    finally:
        S.set_destroy(ctx)
    return out


def _copy_bound(S, js, n, streams, e2e_jobs_per_s, sm_jobs_per_s=None, sm_streams=None):
    """Copy bound of a workload (jobs/s) from pinned copy rates at its mean job sizes, and the
    measured end-to-end rate as a fraction of it: copy engines for the copy-node arms; with
    sm_jobs_per_s also the copy kernels (set_config.sm_copies, measured over sm_streams streams,
    the jobs the arm keeps in flight) and that arm's fraction of its own bound."""
    mi, mo = js.bytes_in // n, js.bytes_out // n

    def bound(rates):
        return max(js.bytes_in / (rates["h2d_gbs"] * 1e9), js.bytes_out / (rates["d2h_gbs"] * 1e9),
                   (js.bytes_in + js.bytes_out) / (rates["bidir_total_gbs"] * 1e9))

    rates = copy_rates(S, mi, mo, streams, reps=1024)
    t = bound(rates)
    out = {"copy_rates_gbs": rates, "mean_in_bytes": mi, "mean_out_bytes": mo, "bound_jobs_per_s": n / t,
           "e2e_frac_of_bound": e2e_jobs_per_s * t / n}
    if sm_jobs_per_s is not None:
        rs = copy_rates(S, mi, mo, sm_streams or streams, reps=1024, sm=True)
        ts = bound(rs)
        out["copy_kernels"] = {"copy_rates_gbs": rs, "streams": sm_streams or streams, "bound_jobs_per_s": n / ts,
                               "sm_copies_frac_of_bound": sm_jobs_per_s * ts / n}
    return out


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def _job_kernel_times(S, js, n, jobs=256):
    """Mean device time (us) of each job's kernel chain launched alone (set_launch_job) on one
    stream, with CUDA events on that stream around every job; a sleep kernel holds the stream
    while the launches are enqueued so the events bracket device time only.  Resident inputs."""
    t = _torch()
    st = t.cuda.Stream()
    sb = max(S.set_job_scratch_bytes(js.kind, S.dims4(*dd)) for dd in js.dims)
    scratch = t.zeros(max(sb, 256), dtype=t.uint8, device="cuda")
    m = min(n, jobs)
    evs = [(t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)) for _ in range(m)]
    with t.cuda.stream(st):
        for k in range(min(m, 8)):  # warm-up
            dd = js.descs_dev[k]
            S.check(S.set_launch_job(ctypes.byref(dd), dd.in_, dd.out, scratch.data_ptr(), k, 0, st.cuda_stream),
                    "set_launch_job")
        st.synchronize()
        t.cuda._sleep(int(2e9 * 40e-6 * m))
        for k in range(m):
            dd = js.descs_dev[k]
            evs[k][0].record(st)
            S.set_launch_job(ctypes.byref(dd), dd.in_, dd.out, scratch.data_ptr(), k, 0, st.cuda_stream)
            evs[k][1].record(st)
    st.synchronize()
    return [a.elapsed_time(b) * 1e3 for a, b in evs], m


def _roofline_hbm(kernel, alg_bytes_per_job, job_us, launches_per_job=1):
    peak = _peaks().get("hbm_gbs", 6800.0)
    ach = alg_bytes_per_job / (job_us * 1e-6) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "alg_bytes_per_job": alg_bytes_per_job, "job_us": job_us, "launches_per_job": launches_per_job,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}


def _eq4(line, bound_jobs_per_s):
    """Eq. 4 schedule fraction 1 - T_ideal / T_measured of every arm of a workload line."""
    return {k: 1 - v["jobs_per_s"] / bound_jobs_per_s for k, v in line.items()
            if isinstance(v, dict) and v.get("jobs_per_s")}


def _kernel_only(S, js, n, launches, flags=0):
    """Profiling: the stage kernels of `launches` resident jobs alone on one stream, then exit."""
    t = _torch()
    sb = max(S.set_job_scratch_bytes(js.kind, S.dims4(*dd)) for dd in js.dims)
    scratch = t.zeros(max(sb, 256), dtype=t.uint8, device="cuda")
    st = t.cuda.current_stream().cuda_stream
    for k in range(launches):
        dd = js.descs_dev[k % n]
        dd.flags |= flags
        S.check(S.set_launch_job(ctypes.byref(dd), dd.in_, dd.out, scratch.data_ptr(), k, 0, st), "set_launch_job")
    t.cuda.synchronize()
    print(json.dumps({"kernel_only": js.kind, "jobs": launches}), flush=True)


def run_copy_rates(args, d: Dist):
    """Pinned host <-> device copy rates (GB/s) by copy size and stream count (set_copy_bandwidth):
    the copy-engine side of every pipeline bound, and the copy kernels of set_config.sm_copies.
    One JSON line per (mover, size, streams)."""
    import paper_2606_05495_gb300 as S
    t = _torch()
    t.cuda.set_device(d.local)
    for mover, base in (("copy_engines", 0), ("copy_kernels", 3)):
        for size in (64 << 10, 128 << 10, 256 << 10, 512 << 10, 2 << 20, 16 << 20, 64 << 20):
            for streams in (1, 4, 8, 16, 32):
                row = {"workload": "copy-rates", "mover": mover, "bytes": size, "streams": streams}
                reps = max(64, min(2048, (512 << 20) // size))
                for name, dirn in (("h2d_gbs", 0), ("d2h_gbs", 1), ("bidir_total_gbs", 2)):
                    g = ctypes.c_double()
                    S.check(S.set_copy_bandwidth(size, streams, reps, base + dirn, ctypes.byref(g)),
                            "set_copy_bandwidth")
                    row[name] = g.value
                if d.rank == 0:
                    print(json.dumps(row), flush=True)


def run_bind_study(args, d: Dist):
    """UpdateGraphParams at dispatch vs at submit (set_config.bind_at_submit) on the scan jobs: one
    JSON line per (io mode, completion mode, dispatch threads, bind)."""
    import paper_2606_05495_gb300 as S
    t = _torch()
    t.cuda.set_device(d.local)
    w = Workload(S, shard(args.jobs, d.rank), d.local)
    nj = len(w.ids)
    for io in (S.SET_IO_HOST, S.SET_IO_DEVICE):
        descs = w.descs_host if io == S.SET_IO_HOST else w.descs_dev
        for cbm, every, workers in ((0, 8, 1), (0, 1, 1), (3, 1, 1), (3, 1, 2), (3, 1, 4)):
            for bind in (0, 1):
                cfg = dict(num_streams=args.streams, num_workers=workers, ring_depth=args.ring, cb_mode=cbm,
                           cb_every=every, device=d.local, io_mode=io, bind_at_submit=bind,
                           slot_bytes=S.set_job_slot_bytes(S.SET_JOB_SAXPY_SCAN_MAX, S.dims4(N_ELEM)))
                ctx = S.create(S.default_config(**cfg))
                ms, st = timed(S, ctx, descs, nj, args, d)
                S.set_destroy(ctx)
                if d.rank == 0:
                    print(json.dumps({"workload": "bind-study", "io": "host" if io == S.SET_IO_HOST else "device",
                                      "cb_mode": cbm, "cb_every": every, "workers": workers, "bind_at_submit": bind,
                                      "jobs_per_s": nj * d.world / (ms * 1e-3), "p99_us": st["p99_us"],
                                      "mean_update_us": st["mean_update_us"], "mean_launch_us": st["mean_launch_us"],
                                      "mean_queue_us": st["mean_queue_us"]}), flush=True)


def run_dd_study(args, d: Dist):
    """Device-dispatch lanes (set_dd) against the host-dispatched executor on the HBM-resident scan
    jobs: one JSON line per lane count and one for the executor."""
    import paper_2606_05495_gb300 as S
    t = _torch()
    t.cuda.set_device(d.local)
    w = Workload(S, shard(args.jobs, d.rank), d.local)
    nj = len(w.ids)
    for streams in (8, 16):
        cfg = dict(num_streams=streams, num_workers=args.workers, ring_depth=args.ring, cb_mode=args.cb_mode,
                   cb_every=args.cb_every, device=d.local, io_mode=S.SET_IO_DEVICE,
                   slot_bytes=S.set_job_slot_bytes(S.SET_JOB_SAXPY_SCAN_MAX, S.dims4(N_ELEM)))
        ctx = S.create(S.default_config(**cfg))
        ms, st = timed(S, ctx, w.descs_dev, nj, args, d)
        S.set_destroy(ctx)
        if d.rank == 0:
            print(json.dumps({"workload": "dd-study", "arm": "executor", "io": "device", "streams": streams,
                              "workers": args.workers, "jobs_per_s": nj * d.world / (ms * 1e-3),
                              "p50_us": st["p50_us"], "p99_us": st["p99_us"],
                              "mean_launch_us": st["mean_launch_us"]}), flush=True)
    for lanes, threads in ((1, 1), (2, 1), (4, 1), (8, 1), (16, 1), (32, 1), (64, 1), (64, 2), (64, 4), (128, 4)):
        arm = device_dispatch_arm(S, w, lanes, d.local, args, d, threads)
        if d.rank == 0:
            print(json.dumps({"workload": "dd-study", "arm": "set_dd", "io": "device", "jobs_per_s": arm["value"],
                              **{k: v for k, v in arm.items() if k not in ("value", "unit", "note")}}), flush=True)


def run_workload(args, d: Dist):
    """One JSON line per workload: SET forms against the batch-synchronous graph baseline."""
    import paper_2606_05495_gb300 as S
    t = _torch()
    t.cuda.set_device(d.local)
    line = {"workload": args.workload, "unit": "jobs/s", "steps": args.steps, "warmup": args.warmup,
            "data": "synthetic (seeded SplitMix64 inputs)"}
    common = dict(num_workers=1, cb_mode=0, device=d.local)
    clocks = Clocks(d.local, args.clock_ms)
    if args.workload == "blur":
        # 64 jobs of 64 KiB last tens of microseconds: a step runs the 64-job configuration 200 times
        # over (12,800 distinct jobs, each with its own input and output)
        n = 64 * 200
        js = JobSet(S, 1, range(n), device_copy=True)
        if args.kernel_only:
            return _kernel_only(S, js, n, args.kernel_only)
        cfg = dict(common, num_streams=2, ring_depth=4, slot_bytes=js.slot_bytes(S))
        line["config"] = {"jobs_per_step": n, "side": 256, "streams": 2, "note": "64-job configuration x 200"}
        polled = dict(cfg, cb_mode=3, num_workers=2)
        line["set"] = _rate(S, polled, js.descs, n, args, d, clocks)
        line["set_host_callbacks_every_8"] = _rate(S, dict(cfg, cb_every=8), js.descs, n, args, d, clocks)
        line["set_host_callbacks_per_job"] = _rate(S, dict(cfg, cb_every=1), js.descs, n, args, d)
        line["set_device_resident"] = _rate(S, dict(polled, io_mode=S.SET_IO_DEVICE), js.descs_dev, n, args, d)
        line["set_16_streams"] = _rate(S, dict(polled, num_streams=16), js.descs, n, args, d)
        line["set_sm_copies"] = _rate(S, dict(polled, sm_copies=1), js.descs, n, args, d)
        line["batch_sync_graph"] = _baseline(S, cfg, S.SET_BASE_BATCH_SYNC, js.descs, n)
        line["single_stream_loop"] = _baseline(S, cfg, S.SET_BASE_SYNC, js.descs, n)
        line["pipeline"] = _copy_bound(S, js, n, 2, line["set"]["jobs_per_s"], line["set_sm_copies"]["jobs_per_s"], 8)
        line["eq4_schedule_frac"] = _eq4(line, line["pipeline"]["bound_jobs_per_s"])
        line["trace"] = _traces(S, polled, js.descs, n)
        ts, m = _job_kernel_times(S, js, n)
        line["roofline"] = _roofline_hbm("blur_hist_kernel", 2 * 65536 + 1040, statistics.mean(ts))
        # kernels reading and writing the pinned buffers over NVLink-C2C, no copy nodes
        line["set_mapped_io"] = _rate(S, dict(polled, io_mode=S.SET_IO_MAPPED), js.descs, n, args, d)
        if not _profiler_attached():
            # HBM-resident blur jobs: the executor (in place) against the device-dispatch lanes, which
            # run queued blur jobs in batches of up to 8 clusters per launch
            alg = 2 * 65536 + 1040
            line["hbm_resident"] = {"jobs": n, "alg_bytes_per_job": alg, "executor_inplace": _rate(
                S, dict(polled, io_mode=S.SET_IO_DEVICE_INPLACE, num_workers=4, num_streams=8), js.descs_dev, n,
                args, d)}
            ddb = S.dd_create(S.dd_default_config(num_lanes=32, device=d.local))
            try:
                ms_dd, st_dd, _ = timed_dd(S, ddb, js.descs_dev, n, args, d)
            finally:
                S.set_dd_destroy(ddb)
            rate = n / (ms_dd * 1e-3)
            line["hbm_resident"]["set_dd_32_lanes"] = {
                "jobs_per_s": rate, "p50_us": st_dd["p50_us"], "p99_us": st_dd["p99_us"], "failed": st_dd["failed"],
                "hbm_frac": rate * alg / 1e9 / _peaks().get("hbm_gbs", 6800.0)}
    elif args.workload in ("img", "mlp"):
        kind = 3 if args.workload == "img" else 4
        n = min(args.jobs, 2000)
        js = JobSet(S, kind, range(n), device_copy=bool(args.kernel_only))
        if args.kernel_only:
            return _kernel_only(S, js, n, args.kernel_only, S.SET_F_PER_STAGE if args.per_stage else 0)
        sb = js.slot_bytes(S)
        cfg = dict(common, num_streams=16, ring_depth=4, slot_bytes=sb)
        line["config"] = {"jobs": n, "sample_of": 10000 if kind == 3 else 2000, "streams": 16,
                          "in_bytes": js.bytes_in, "out_bytes": js.bytes_out}
        polled = dict(cfg, cb_mode=3, num_workers=2)
        line["set_per_job"] = _rate(S, polled, js.descs, n, args, d, clocks)
        line["set_per_job_host_callbacks"] = _rate(S, dict(cfg, cb_every=8), js.descs, n, args, d, clocks)
        if kind == 3:
            line["set_per_stage_graphs"] = _rate(S, dict(polled, img_fused=0), js.descs, n, args, d)
        line["set_per_job_sm_copies"] = _rate(S, dict(polled, sm_copies=1), js.descs, n, args, d)
        # batched form: autotuned jobs per launch (and tile / CTAs per SM for images) in an 8 GiB arena
        # polled completion: a batch launch's host-callback chain would cost more than its copies
        bcfg = dict(cfg, cb_mode=3, ring_depth=2, batch_max=16, arena_bytes=8 << 30, slot_bytes=1 << 30)
        ctx = S.create(S.default_config(**bcfg))
        tune = S.set_tune_result()
        ns = min(n, 64)
        S.check(S.set_autotune(ctx, kind, js.descs, ns, ctypes.byref(tune)), "set_autotune", ctx)
        ms, st = timed(S, ctx, js.descs, n, args, d, clocks)
        S.set_destroy(ctx)
        line["set_batched"] = {"jobs_per_s": n / (ms * 1e-3), "ms_per_step": ms, "p99_us": st["p99_us"],
                               "failed": st["failed"], "autotune": tune.as_dict()}
        line["batch_sync_graph"] = _baseline(S, cfg, S.SET_BASE_BATCH_SYNC, js.descs, n)
        best = max(line["set_per_job"]["jobs_per_s"], line["set_batched"]["jobs_per_s"])
        line["pipeline"] = _copy_bound(S, js, n, 16, best, line["set_per_job_sm_copies"]["jobs_per_s"], 64)
        line["eq4_schedule_frac"] = _eq4(line, line["pipeline"]["bound_jobs_per_s"])
        line["trace"] = _traces(S, polled, js.descs, n)
        dev = JobSet(S, kind, range(min(n, 256)), device_copy=True)  # resident copies for the kernels alone
        if kind == 3 and not _profiler_attached():
            # HBM-resident image jobs: the executor (in place) against the device-dispatch lanes
            nd = len(dev.ids)
            line["hbm_resident"] = {"jobs": nd, "executor_inplace": _rate(
                S, dict(polled, io_mode=S.SET_IO_DEVICE_INPLACE, num_workers=4), dev.descs_dev, nd, args, d)}
            ddh = S.dd_create(S.dd_default_config(num_lanes=16, device=d.local))
            try:
                ms_dd, st_dd, _ = timed_dd(S, ddh, dev.descs_dev, nd, args, d)
            finally:
                S.set_dd_destroy(ddh)
            line["hbm_resident"]["set_dd_16_lanes"] = {"jobs_per_s": nd / (ms_dd * 1e-3), "p99_us": st_dd["p99_us"],
                                                       "failed": st_dd["failed"]}
        ts, m = _job_kernel_times(S, dev, len(dev.ids))
        if kind == 3:
            px = [W * H for (W, H) in dev.dims[:m]]
            alg = statistics.mean(4 * p + 1040 for p in px)  # read RGB, write Sobel + histogram
            line["roofline"] = _roofline_hbm("img_fused_kernel", alg, statistics.mean(ts))
        else:
            rows = [dd[0] for dd in dev.dims[:m]]
            flop = statistics.mean(2 * 2 * r * 1024 * 4096 for r in rows)
            pk = _peaks().get("bf16_tflops", 1900.0)
            ach = flop / (statistics.mean(ts) * 1e-6) / 1e12
            line["roofline"] = {"bound": "tensor", "kernel": "mlp_gemm_kernel (+ layernorm_kernel)", "achieved": ach,
                                "peak": pk, "unit": "TFLOP/s", "frac": ach / pk, "flop_per_job": flop,
                                "job_us": statistics.mean(ts), "launches_per_job": 3,
                                "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)"}
        if kind == 4:
            flop = 2.0 * js.rows() * 1024 * 4096 * 2
            line["gemm_tflops_e2e"] = {k: flop / (line[k]["ms_per_step"] * 1e-3) / 1e12
                                       for k in ("set_per_job", "set_batched")}
    elif args.workload == "hot":
        # hotspot: 512 x 512 cells, 64 steps per job (8 temporally blocked launches of 8 steps)
        n = min(args.jobs, 1000)
        js = JobSet(S, 5, range(n), device_copy=True)
        C, R, K = js.dims[0]
        if args.kernel_only:
            return _kernel_only(S, js, n, args.kernel_only)
        cfg = dict(common, num_streams=16, ring_depth=4, slot_bytes=js.slot_bytes(S))
        line["config"] = {"jobs": n, "grid": [R, C], "steps": K, "streams": 16, "in_bytes": js.bytes_in,
                          "out_bytes": js.bytes_out, "l2": "inputs > L2 (no flush needed)"}
        line["set_cb_every_8"] = _rate(S, dict(cfg, cb_every=8), js.descs, n, args, d, clocks)
        line["set_polled_2_workers"] = _rate(S, dict(cfg, cb_mode=3, num_workers=2), js.descs, n, args, d, clocks)
        line["set_sm_copies"] = _rate(S, dict(cfg, cb_mode=3, num_workers=2, sm_copies=1), js.descs, n, args, d)
        line["set_device_resident"] = _rate(S, dict(cfg, cb_mode=3, num_workers=2, io_mode=S.SET_IO_DEVICE),
                                            js.descs_dev, n, args, d, clocks)
        line["batch_sync_graph"] = _baseline(S, cfg, S.SET_BASE_BATCH_SYNC, js.descs, n)
        line["single_stream_loop"] = _baseline(S, cfg, S.SET_BASE_SYNC, js.descs, n)
        line["pipeline"] = _copy_bound(S, js, n, 16, line["set_polled_2_workers"]["jobs_per_s"])
        line["eq4_schedule_frac"] = _eq4(line, line["pipeline"]["bound_jobs_per_s"])
        line["trace"] = _traces(S, dict(cfg, cb_mode=3, num_workers=2), js.descs, n)
        # the kernel chain alone: CUDA events around each job's 8 launches on one stream
        st = t.cuda.Stream()
        scratch = t.zeros(S.set_job_scratch_bytes(5, S.dims4(C, R, K)), dtype=t.uint8, device="cuda")
        m = min(n, 256)
        evs = [(t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)) for _ in range(m)]
        with t.cuda.stream(st):
            for k in range(8):
                dd = js.descs_dev[k]
                S.check(S.set_launch_job(ctypes.byref(dd), dd.in_, dd.out, scratch.data_ptr(), k, 0, st.cuda_stream),
                        "launch")
            st.synchronize()
            t.cuda._sleep(int(2e9 * 60e-6 * m))  # hold the stream while the launches are enqueued
            for k in range(m):
                dd = js.descs_dev[k]
                evs[k][0].record(st)
                S.set_launch_job(ctypes.byref(dd), dd.in_, dd.out, scratch.data_ptr(), k, 0, st.cuda_stream)
                evs[k][1].record(st)
        st.synchronize()
        job_us = statistics.mean(a.elapsed_time(b) * 1e3 for a, b in evs)
        launch_us = job_us / 8
        alg = 12 * R * C  # per launch: read T and P, write T
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except OSError:
            pass
        peak = peaks.get("hbm_gbs", 6800.0)
        line["roofline"] = {"bound": "hbm", "kernel": "hotspot_kernel", "achieved": alg / (launch_us * 1e-6) / 1e9,
                            "peak": peak, "unit": "GB/s", "frac": alg / (launch_us * 1e-6) / 1e9 / peak,
                            "alg_bytes_per_launch": alg, "launch_us": launch_us, "job_us": job_us,
                            "cell_steps_per_s": R * C * K / (job_us * 1e-6)}
    elif args.workload == "serve":
        import numpy as np

        import datagen
        npool = args.jobs if args.jobs != 4096 else 2000
        rates = [float(r) for r in args.rates.split(",")]
        pools = {}
        for lam in rates[:1]:
            _, kinds, _ = datagen.serve_trace(lam, npool)
        counts = {k: int((kinds == k).sum() * 1.15) + 16 for k in (1, 3, 4)}  # traces of other rates vary
        for k in (1, 3, 4):
            pools[k] = JobSet(S, k, range(50000 + 100000 * k, 50000 + 100000 * k + counts[k]))
        cfg = dict(common, num_streams=16, ring_depth=4, cb_every=1, slot_bytes=64 << 20, arena_bytes=8 << 30)
        line["config"] = {"arrivals_per_rate": npool, "mix": "40% blur 256x256, 40% image (log-uniform sides), "
                          "20% MLP (m 1..256)", "arena_bytes": 8 << 30, "streams": 16, "ring_depth": 4,
                          "workers": "2 (polled arms), 1 (host-callback arm)"}
        sweep = []
        for lam in rates:
            ts, kinds, _ = datagen.serve_trace(lam, npool)
            used = {1: 0, 3: 0, 4: 0}
            arr = (S.set_job_desc * npool)()
            for i, k in enumerate(kinds):
                arr[i] = pools[int(k)].descs[used[int(k)] % len(pools[int(k)].ids)]
                used[int(k)] += 1
            off = (ctypes.c_uint64 * npool)(*[int(x * 1e9) for x in ts])
            row = {"rate": lam}
            # set: the request loop binds and launches an arrival itself when a slot and its memory
            # are free (bind_at_submit 2; otherwise a dispatch thread does when one frees up),
            # completion by the polling thread (cb_mode 3); set_dispatch_threads: every arrival is
            # queued and launched by a dispatch thread; set_host_callbacks: that, with Algorithm 3's
            # host function on the lane stream (cb_mode 1); set_continuous_batching: dispatch threads
            # pack the image and MLP arrivals queued at that moment into one batched launch (up to 16)
            # set_sm_copies: "set" with the copies done by copy kernels (set_config.sm_copies)
            for name, mode, cbm, bind, nw, bmax, smc in (("set", S.SET_SERVE_SET, 3, 2, 2, 1, 0),
                                                         ("set_sm_copies", S.SET_SERVE_SET, 3, 2, 2, 1, 1),
                                                         ("set_dispatch_threads", S.SET_SERVE_SET, 3, 0, 2, 1, 0),
                                                         ("set_continuous_batching", S.SET_SERVE_SET, 3, 0, 2, 16, 0),
                                                         ("set_host_callbacks", S.SET_SERVE_SET, 1, 0, 1, 1, 0),
                                                         ("batch_sync_graph", S.SET_SERVE_BATCH_SYNC, 1, 0, 1, 1, 0)):
                ctx = S.create(S.default_config(**dict(cfg, cb_mode=cbm, bind_at_submit=bind, num_workers=nw,
                                                       batch_max=bmax, sm_copies=smc)))
                st = S.set_stats_t()
                with clocks.window():
                    S.check(S.set_serve(ctx, mode, arr, off, npool, ctypes.byref(st)), "set_serve", ctx)
                S.set_destroy(ctx)
                row[name] = {"jobs_per_s": st.jobs_per_s, "p50_us": st.p50_us, "p99_us": st.p99_us,
                             "failed": st.failed, "mem_waits": st.mem_waits}
                if mode == S.SET_SERVE_SET:
                    row[name].update(queue_us=st.mean_queue_us, service_us=st.mean_service_us)
            sweep.append(row)
            print(json.dumps(row), flush=True)
        line["sweep"] = sweep
    line["clocks"] = clocks.stop()
    if d.rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    d = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, d)
        elif args.workload == "bind-study":
            run_bind_study(args, d)
        elif args.workload == "copy-rates":
            run_copy_rates(args, d)
        elif args.workload == "dd-study":
            run_dd_study(args, d)
        elif args.workload != "scan":
            run_workload(args, d)
        else:
            run_set(args, d)
    finally:
        d.close()


if __name__ == "__main__":
    main()
