"""The C ABI on CPU: libset.so loads, exports every function include/set.h declares, the Python
structs match the C layouts, and the documented payload sizes hold.  No compute calls."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_2606_05495_gb300 as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "set.h")


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(set_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_function_is_exported():
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(S.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    nm = subprocess.run(["nm", "-D", "--defined-only", S.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (set_\w+)", nm))
    assert set(names) <= exported


STRUCTS = {
    "set_job_desc": S.set_job_desc,
    "set_config": S.set_config,
    "set_stats_t": S.set_stats_t,
    "set_trailer": S.set_trailer,
    "set_trace_summary": S.set_trace_summary,
    "set_tune_result": S.set_tune_result,
    "set_dd_config": S.set_dd_config,
}


def test_struct_layouts_match_binding():
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "set.h"', "int main(void){"]
    for cname, py in STRUCTS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            cf = "in" if fname == "in_" else fname
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {cf}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        cname, field, val = line.split()
        py = STRUCTS[cname]
        got = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert got == int(val), (cname, field, got, val)


def test_documented_payload_sizes():
    d = S.dims4
    assert S.set_job_in_bytes(1, d(256, 256)) == 65536
    assert S.set_job_out_bytes(1, d(256, 256)) == 65536 + 1024 + 16
    assert S.set_job_out_bytes(1, d(17, 3)) == 64 + 1024 + 16  # 51 bytes padded to 64
    assert S.set_job_in_bytes(2, d(65536)) == 524288
    assert S.set_job_out_bytes(2, d(65536)) == 524288 + 32
    assert S.set_job_in_bytes(3, d(640, 480)) == 640 * 480 * 3
    assert S.set_job_out_bytes(3, d(641, 3)) == 1936 + 1024 + 16
    assert S.set_job_in_bytes(4, d(7)) == 7 * 1024 * 2
    assert S.set_job_out_bytes(4, d(7)) == 7 * 1024 * 4 + 16
    assert S.set_job_in_bytes(5, d(512, 512, 64)) == 2 * 512 * 512 * 4  # T0 then P
    assert S.set_job_out_bytes(5, d(512, 512, 64)) == 512 * 512 * 4 + 16
    assert S.set_job_out_bytes(5, d(3, 5, 1)) == 64 + 16  # 60 bytes padded to 64
    for t, dims in [(1, d(0, 5)), (1, d(2049, 5)), (2, d(0)), (2, d(1 << 27)), (3, d(4097, 2)), (4, d(0)),
                    (4, d(257)), (5, d(16, 16, 0)), (5, d(16, 16, 65)), (5, d(8193, 2, 1)), (9, d(1, 1))]:
        assert S.set_job_in_bytes(t, dims) == 0 and S.set_job_out_bytes(t, dims) == 0
    assert S.set_job_scratch_bytes(2, d(65536)) == 512  # 64-byte header + 16 tiles x 16 bytes, aligned
    sb = S.set_job_slot_bytes(2, d(65536))
    assert sb >= 2 * 524288 and sb < 2 * 524288 + 4096


def test_config_defaults():
    c = S.default_config()
    assert (c.num_streams, c.num_workers, c.ring_depth, c.queue_capacity, c.steal) == (2, 2, 2, 4, 1)
    assert c.io_mode == S.SET_IO_HOST and c.img_fused == 1 and c.drain_timeout_ms == 30000


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = ctypes.c_void_p()
    assert S.set_create(2, 2, 1 << 20, ctypes.byref(ctx)) == S.SET_ECUDA
    assert S.set_last_error(None)
    assert S.set_submit(None, None, None) == S.SET_EINVAL


def test_dd_config_defaults_and_validation_without_gpu():
    c = S.dd_default_config()
    assert (c.num_lanes, c.ring_depth, c.scan_max_n, c.blur_max_w, c.idle_us) == (16, 64, 65536, 256, 2000)
    dd = ctypes.c_void_p()
    # configuration is checked before any CUDA call
    for bad in (dict(num_lanes=0), dict(ring_depth=0), dict(scan_max_n=0), dict(scan_max_n=(1 << 26) + 1),
                dict(blur_max_w=2049), dict(idle_us=0)):
        assert S.set_dd_create(ctypes.byref(S.dd_default_config(**bad)), ctypes.byref(dd)) == S.SET_EINVAL
        assert not dd.value and S.set_dd_last_error(None)
    assert S.set_dd_submit(None, None, None) == S.SET_EINVAL
    assert S.set_dd_wait_all(None, 0) == S.SET_EINVAL
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert S.set_dd_create(ctypes.byref(c), ctypes.byref(dd)) == S.SET_ECUDA and not dd.value


def test_sm_copies_configurations_refused_without_gpu():
    # checked before any CUDA call: copy kernels only for pinned host I/O of per-job graphs
    assert S.default_config().sm_copies == 0
    ctx = ctypes.c_void_p()
    for bad in (dict(io_mode=S.SET_IO_DEVICE), dict(io_mode=S.SET_IO_MAPPED_IN), dict(batch_max=4), dict(sm_copies=-1)):
        cfg = S.default_config(**dict(dict(sm_copies=1), **bad))
        assert S.set_create_ex(ctypes.byref(cfg), ctypes.byref(ctx)) == S.SET_EINVAL
        assert b"sm_copies" in S.set_last_error(None)


def test_copy_bandwidth_arguments_checked_without_gpu():
    g = ctypes.c_double()
    for args in ((0, 8, 16, 0), (1 << 20, 0, 16, 0), (1 << 20, 8, 0, 3), (1 << 20, 8, 16, 6), (1 << 20, 8, 16, -1)):
        assert S.set_copy_bandwidth(*args, ctypes.byref(g)) == S.SET_EINVAL
    assert S.set_copy_bandwidth(1 << 20, 8, 16, 0, None) == S.SET_EINVAL
