"""Python binding of the SET executor's C ABI (include/set.h): argument marshalling only.

Every name below is the C function or struct of the same name; the work runs in
lib/libset.so (host runtime + sm_103a stage kernels).  Importing this package
fails loudly if the library has not been built (``build.build()`` or
``__graft_entry__.build()``); there is no fallback path.

Host buffers passed as ``in_`` / ``out`` must be page-locked (for example
``torch.empty(n, dtype=torch.uint8, pin_memory=True)``); device buffers (with
SET_IO_DEVICE) are plain CUDA pointers such as ``tensor.data_ptr()``.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_int32, c_int64, c_size_t, c_uint32, c_uint64, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libset.so")

SET_OK, SET_EINVAL, SET_ENOMEM, SET_EAGAIN, SET_ETIMEDOUT, SET_ECUDA, SET_ESHUTDOWN, SET_EDEVICE = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "SET_OK", -1: "SET_EINVAL", -2: "SET_ENOMEM", -3: "SET_EAGAIN", -4: "SET_ETIMEDOUT",
                -5: "SET_ECUDA", -6: "SET_ESHUTDOWN", -7: "SET_EDEVICE"}
SET_JOB_BLUR_HIST, SET_JOB_SAXPY_SCAN_MAX, SET_JOB_IMG_SOBEL_HIST, SET_JOB_MLP_LN, SET_JOB_HOTSPOT = 1, 2, 3, 4, 5
SET_F_NONBLOCK = 0x1
SET_F_PER_STAGE = 0x2
SET_F_TEST_STALL = 0x100
SET_F_TEST_GUARD = 0x200
SET_IO_HOST, SET_IO_DEVICE, SET_IO_MAPPED, SET_IO_MAPPED_IN, SET_IO_MAPPED_OUT, SET_IO_DEVICE_INPLACE = 0, 1, 2, 3, 4, 5
SET_BASE_SYNC, SET_BASE_BATCH_SYNC = 1, 2
SET_SERVE_SET, SET_SERVE_BATCH_SYNC = 0, 1
SET_TRAILER_MAGIC = 0x5E7C
SET_DEVERR_WAIT = 0x1
SET_DEVERR_GUARD = 0x2


class set_trailer(ctypes.Structure):
    _fields_ = [("job_id", c_uint64), ("slot_gen", c_uint32), ("word", c_uint32)]


class set_job_desc(ctypes.Structure):
    # "in" is a Python keyword: the field is spelled in_ here
    _fields_ = [("type", c_uint32), ("flags", c_uint32), ("in_", c_void_p), ("in_bytes", c_size_t),
                ("out", c_void_p), ("out_bytes", c_size_t), ("dims", c_uint32 * 4), ("scalar", c_float),
                ("reserved", c_uint32), ("shared", c_void_p * 2), ("user_tag", c_uint64),
                ("t_arrival_ns", c_uint64), ("status", POINTER(c_int32))]


class set_config(ctypes.Structure):
    _fields_ = [("num_streams", c_int), ("num_workers", c_int), ("slot_bytes", c_size_t), ("ring_depth", c_int),
                ("queue_capacity", c_int), ("steal", c_int), ("io_mode", c_int), ("img_fused", c_int),
                ("pool", c_void_p), ("pool_bytes", c_size_t), ("type_mask", c_uint32), ("device", c_int),
                ("drain_timeout_ms", c_int), ("cb_mode", c_int), ("spin_us", c_int), ("cb_every", c_int),
                ("batch_max", c_int), ("img_ctas_per_sm", c_int), ("img_tile", c_int), ("stamps", c_int),
                ("arena_bytes", c_size_t), ("bind_at_submit", c_int), ("guards", c_int), ("sm_copies", c_int)]


class set_stats_t(ctypes.Structure):
    _fields_ = [("submitted", c_uint64), ("completed", c_uint64), ("failed", c_uint64), ("steals", c_uint64),
                ("updates", c_uint64), ("canary_errors", c_uint64), ("elapsed_s", c_double),
                ("jobs_per_s", c_double), ("p50_us", c_double), ("p99_us", c_double), ("max_us", c_double),
                ("mean_update_us", c_double), ("mean_launch_us", c_double), ("mem_waits", c_uint64),
                ("order_errors", c_uint64), ("arena_peak_bytes", c_uint64),
                ("mean_queue_us", c_double), ("mean_service_us", c_double), ("mean_kernel_gap_us", c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class set_trace_summary(ctypes.Structure):
    _fields_ = [("kernels", c_uint64), ("memcpys", c_uint64), ("span_us", c_double), ("kernel_busy_us", c_double),
                ("copy_busy_us", c_double), ("any_busy_us", c_double), ("idle_frac", c_double),
                ("mean_kernel_gap_us", c_double), ("max_kernel_gap_us", c_double), ("top_kernel", ctypes.c_char * 128),
                ("top_kernel_launches", c_uint64), ("top_kernel_mean_us", c_double), ("top_kernel_share", c_double)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["top_kernel"] = self.top_kernel.decode(errors="replace")
        return d


class set_tune_result(ctypes.Structure):
    _fields_ = [("batch_max", c_int), ("img_tile", c_int), ("img_ctas_per_sm", c_int), ("candidates", c_int),
                ("jobs_per_s", c_double), ("single_jobs_per_s", c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class set_dd_config(ctypes.Structure):
    _fields_ = [("num_lanes", c_int), ("ring_depth", c_int), ("device", c_int), ("scan_max_n", c_uint32),
                ("blur_max_w", c_uint32), ("idle_us", c_int), ("spin_us", c_int), ("drain_timeout_ms", c_int)]


class SetError(RuntimeError):
    def __init__(self, status: int, where: str, text: str = ""):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {text}".strip())
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2606_05495_gb300/build.py` "
                      "(or __graft_entry__.build()); there is no fallback implementation")

_lib = ctypes.CDLL(LIB_PATH)
_dims = POINTER(c_uint32)
_SIGS = {
    "set_job_in_bytes": ([c_uint32, _dims], c_size_t),
    "set_job_out_bytes": ([c_uint32, _dims], c_size_t),
    "set_job_scratch_bytes": ([c_uint32, _dims], c_size_t),
    "set_job_slot_bytes": ([c_uint32, _dims], c_size_t),
    "set_config_default": ([POINTER(set_config)], None),
    "set_create": ([c_int, c_int, c_size_t, POINTER(c_void_p)], c_int),
    "set_create_ex": ([POINTER(set_config), POINTER(c_void_p)], c_int),
    "set_submit": ([c_void_p, POINTER(set_job_desc), POINTER(c_uint64)], c_int),
    "set_submit_many": ([c_void_p, POINTER(set_job_desc), c_size_t, POINTER(c_uint64), POINTER(c_size_t)], c_int),
    "set_wait_all": ([c_void_p, c_int64], c_int),
    "set_stats": ([c_void_p, POINTER(set_stats_t)], c_int),
    "set_reset_stats": ([c_void_p], c_int),
    "set_destroy": ([c_void_p], c_int),
    "set_last_error": ([c_void_p], c_char_p),
    "set_launch_job": ([POINTER(set_job_desc), c_void_p, c_void_p, c_void_p, c_uint64, c_uint32, c_void_p], c_int),
    "set_job_kernel_count": ([c_uint32, _dims, c_int], c_int),
    "set_launch_scan_static": ([POINTER(set_job_desc), c_void_p, c_void_p, c_uint64, c_uint32, c_void_p], c_int),
    "set_run_baseline": ([c_void_p, c_int, POINTER(set_job_desc), c_size_t, POINTER(set_stats_t)], c_int),
    "set_copy_bandwidth": ([c_size_t, c_int, c_int, c_int, POINTER(c_double)], c_int),
    "set_trace_start": ([], c_int),
    "set_autotune": ([c_void_p, c_uint32, POINTER(set_job_desc), c_size_t, POINTER(set_tune_result)], c_int),
    "set_serve": ([c_void_p, c_int, POINTER(set_job_desc), POINTER(c_uint64), c_size_t, POINTER(set_stats_t)], c_int),
    "set_trace_stop": ([POINTER(set_trace_summary)], c_int),
    "set_dd_config_default": ([POINTER(set_dd_config)], None),
    "set_dd_create": ([POINTER(set_dd_config), POINTER(c_void_p)], c_int),
    "set_dd_submit": ([c_void_p, POINTER(set_job_desc), POINTER(c_uint64)], c_int),
    "set_dd_submit_many": ([c_void_p, POINTER(set_job_desc), c_size_t, POINTER(c_uint64), POINTER(c_size_t)], c_int),
    "set_dd_wait_all": ([c_void_p, c_int64], c_int),
    "set_dd_stats": ([c_void_p, POINTER(set_stats_t), POINTER(c_uint64)], c_int),
    "set_dd_reset_stats": ([c_void_p], c_int),
    "set_dd_destroy": ([c_void_p], c_int),
    "set_dd_last_error": ([c_void_p], c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes, _fn.restype = _args, _res
    globals()[_name] = _fn


def dims4(*d) -> "ctypes.Array":
    a = (c_uint32 * 4)()
    for i, v in enumerate(d):
        a[i] = int(v)
    return a


def check(status: int, where: str, ctx=None) -> None:
    """Raises SetError with set_last_error's text unless status is SET_OK."""
    if status != SET_OK:
        txt = set_last_error(ctx)
        raise SetError(status, where, txt.decode() if txt else "")


def make_desc(type_: int, dims, in_ptr: int, out_ptr: int, scalar: float = 0.0, shared=(None, None),
              flags: int = 0, user_tag: int = 0, t_arrival_ns: int = 0, status=None) -> set_job_desc:
    """Fills a set_job_desc; in/out byte counts come from set_job_in_bytes / set_job_out_bytes."""
    d = set_job_desc()
    d.type = type_
    d.flags = flags
    dd = dims4(*dims)
    d.dims = dd
    d.in_ = in_ptr
    d.in_bytes = set_job_in_bytes(type_, dd)
    d.out = out_ptr
    d.out_bytes = set_job_out_bytes(type_, dd)
    d.scalar = scalar
    d.shared[0] = shared[0]
    d.shared[1] = shared[1]
    d.user_tag = user_tag
    d.t_arrival_ns = t_arrival_ns
    if status is not None:
        d.status = status
    return d


def create(cfg: set_config) -> c_void_p:
    """set_create_ex that raises on failure; returns the context handle."""
    ctx = c_void_p()
    check(set_create_ex(ctypes.byref(cfg), ctypes.byref(ctx)), "set_create_ex")
    return ctx


def default_config(**kw) -> set_config:
    c = set_config()
    set_config_default(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def dd_default_config(**kw) -> set_dd_config:
    c = set_dd_config()
    set_dd_config_default(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def dd_check(status: int, where: str, dd=None) -> None:
    """check() for the device-dispatch object (set_dd_last_error's text)."""
    if status != SET_OK:
        txt = set_dd_last_error(dd)
        raise SetError(status, where, txt.decode() if txt else "")


def dd_create(cfg: set_dd_config) -> c_void_p:
    """set_dd_create that raises on failure; returns the handle."""
    dd = c_void_p()
    dd_check(set_dd_create(ctypes.byref(cfg), ctypes.byref(dd)), "set_dd_create")
    return dd
