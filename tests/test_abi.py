"""The C ABI: libmpx.so loads on a machine without a GPU driver and exports
every function include/mpx.h declares; calls that need a GPU fail with an
error code instead of crashing."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\bint\s+(mpx_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = os.path.join(ROOT, "paper_2208_13707_gb300", "_lib", "libmpx.so")
    if not os.path.exists(path):
        from paper_2208_13707_gb300 import build
        build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ["mpx_stream_create", "mpx_stream_free", "mpx_stream_comm_create", "mpx_send_enqueue",
              "mpx_recv_enqueue", "mpx_isend_enqueue", "mpx_irecv_enqueue", "mpx_wait_enqueue",
              "mpx_waitall_enqueue", "mpx_allreduce_enqueue", "mpx_type_vector"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert missing == []


def test_binding_exposes_the_same_names():
    from paper_2208_13707_gb300 import mpx
    missing = [n for n in _declared() if not hasattr(mpx, n)]
    assert missing == []


def test_datatype_calls_work_without_a_gpu():
    from paper_2208_13707_gb300 import mpx
    t = mpx.mpx_type_vector(4, 2, 3, mpx.FLOAT)
    assert mpx.mpx_type_size(t) == 4 * 2 * 4
    assert mpx.mpx_type_extent(t) == ((4 - 1) * 3 + 2) * 4
    st = mpx.Status(source=1, tag=2, error=0, pad=0, bytes=20)
    assert mpx.mpx_get_count(st, mpx.INT32) == 5
    assert mpx.mpx_get_count(st, mpx.INT64) == mpx.UNDEFINED
    mpx.mpx_type_free(t)
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_type_vector(0, 1, 1, mpx.FLOAT)
    assert e.value.code == mpx.ERR_ARG
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_type_vector(2, 3, 2, mpx.FLOAT)        # stride < blocklength
    assert e.value.code == mpx.ERR_ARG


def test_world_create_reports_missing_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2208_13707_gb300 import mpx
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_world_create(2)
    assert e.value.code == mpx.ERR_CUDA


def test_config_defaults_and_validation():
    from paper_2208_13707_gb300 import mpx
    c = mpx.mpx_world_config_init()
    assert c.ring_slots & (c.ring_slots - 1) == 0
    assert c.engine_threads % 32 == 0 and c.engine_threads <= 512
    assert c.watchdog_ns > 0 and c.staging_bytes > 0
    bad = mpx.mpx_world_config_init()
    bad.ring_slots = 1000                                # not a power of two
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_world_create(2, bad)
    assert e.value.code == mpx.ERR_ARG
    # submission rings in pinned host memory unless asked otherwise; an unknown
    # placement is refused before any CUDA call
    assert c.ring_placement == mpx.RINGS_HOST and c.reserved0 == 0
    bad = mpx.mpx_world_config_init()
    bad.ring_placement = 7
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_world_create(2, bad)
    assert e.value.code == mpx.ERR_ARG


def test_diagnostic_entry_points_are_bound():
    """The engine trace and the device-attribute query are diagnostics of the
    library (not part of the header's API): bound, and without a world the
    trace is empty."""
    from paper_2208_13707_gb300 import mpx
    assert callable(mpx.engine_trace) and callable(mpx.device_attr)
    assert mpx.lib.mpxi_world_trace(None, None, 0) == 0


def test_sendrecv_static_rejects_bad_arguments_before_touching_the_gpu():
    from paper_2208_13707_gb300 import mpx
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_sendrecv_static(0, 1, 999, 0, 1, mpx.FLOAT, 0)
    assert e.value.code == mpx.ERR_TYPE
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_sendrecv_static(16, 5 << 20, mpx.FLOAT, 32, 5 << 20, mpx.FLOAT, 0)
    assert e.value.code == mpx.ERR_NO_MEM


def test_byte_spans_that_would_overflow_are_rejected():
    """Byte counts are products of counts, vector shapes and element sizes;
    spans beyond 2^60 bytes are refused with MPX_ERR_ARG before any product is
    formed (a wrapped count could otherwise look small)."""
    from paper_2208_13707_gb300 import mpx
    with pytest.raises(mpx.MpxError) as e:       # one instance spans about 2^62 bytes
        mpx.mpx_type_vector(1 << 30, 1, 1 << 30, mpx.FLOAT)
    assert e.value.code == mpx.ERR_ARG
    big = mpx.mpx_type_vector(1 << 16, 1, 1 << 20, mpx.DOUBLE)  # 2^39-byte extent: accepted
    try:
        for cnt in ((1 << 62), (1 << 40)):        # 2^62 * 8 and 2^40 * 2^39 bytes
            ty = mpx.DOUBLE if cnt == (1 << 62) else big
            with pytest.raises(mpx.MpxError) as e:
                mpx.mpx_sendrecv_static(16, cnt, ty, 32, 1, mpx.BYTE, 0)
            assert e.value.code == mpx.ERR_ARG
            with pytest.raises(mpx.MpxError) as e:
                mpx.mpx_sendrecv_static(16, 1, mpx.BYTE, 32, cnt, ty, 0)
            assert e.value.code == mpx.ERR_ARG
    finally:
        mpx.mpx_type_free(big)


def test_op_struct_layout_matches_the_binding(tmp_path):
    """mpx_op_t as the C compiler lays it out equals the binding's numpy layout."""
    from paper_2208_13707_gb300 import mpx
    dt = mpx.op_dtype()
    fields = list(dt.names)
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mpx.h"\nint main(void){\n'
                   '  printf("%zu", sizeof(mpx_op_t));\n' +
                   "".join(f'  printf(" %zu", offsetof(mpx_op_t, {f}));\n' for f in fields) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == dt.itemsize
    assert out[1:] == [dt.fields[f][1] for f in fields]


def test_serve_call_layout_matches_the_binding(tmp_path):
    """mpx_serve_call_t as the C compiler lays it out equals the numpy layout
    the binding and the schedule generator use."""
    import subprocess
    from paper_2208_13707_gb300 import mpx
    from traffic.gen import SERVE_CALL_DTYPE
    dt = mpx.serve_call_dtype()
    assert dt == SERVE_CALL_DTYPE
    fields = list(dt.names)
    src = tmp_path / "call.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mpx.h"\nint main(void){\n'
                   '  printf("%zu", sizeof(mpx_serve_call_t));\n' +
                   "".join(f'  printf(" %zu", offsetof(mpx_serve_call_t, {f}));\n' for f in fields) +
                   "  return 0;\n}\n")
    exe = tmp_path / "call"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == dt.itemsize
    assert out[1:] == [dt.fields[f][1] for f in fields]
    assert (mpx.SERVE_SEND, mpx.SERVE_RECV, mpx.SERVE_WAITALL, mpx.SERVE_ALLREDUCE) == (0, 1, 2, 3)


def test_serve_schedule_rejects_out_of_range_calls():
    """Schedule checks run before any GPU work: a peer outside the threads,
    an offset past the region, a capture past the capture area."""
    import numpy as np
    from paper_2208_13707_gb300 import mpx
    c = mpx.mpx_serve_config_init()
    c.nthreads = 2
    calls = np.zeros(2, mpx.serve_call_dtype())
    calls["kind"] = [mpx.SERVE_SEND, mpx.SERVE_RECV]
    calls["peer"] = [1, 0]
    calls["bytes"] = 64
    calls["capture"] = -1
    lo = np.array([0, 1, 2], np.int64)
    bad = [("peer", 0, 2), ("off", 0, 4050), ("capture", 1, 64)]
    for field, i, v in bad:
        x = calls.copy()
        x[field][i] = v
        with pytest.raises(mpx.MpxError) as e:
            mpx.mpx_serve_run_schedule(c, x, lo, [64, 128], 4096, capture=256, capture_bytes=64)
        assert e.value.code == mpx.ERR_ARG, field


def test_enqueue_batch_stops_at_the_first_invalid_op():
    """Validation happens before anything is published: an op without a
    communicator fails with MPX_ERR_COMM and nothing counts as enqueued."""
    import numpy as np
    from paper_2208_13707_gb300 import mpx
    ops = np.zeros(3, mpx.op_dtype())
    ops["kind"] = mpx.OP_SEND
    ops["count"] = 1
    ops["buf"] = 64
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_enqueue_batch(ops)
    assert e.value.code == mpx.ERR_COMM and e.value.done == 0
    ops["kind"] = 99
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_enqueue_batch(ops)
    assert e.value.code == mpx.ERR_ARG and e.value.done == 0
    assert mpx.mpx_enqueue_batch(ops[:0]) == 0


@pytest.mark.parametrize("cname,pyname", [("mpx_serve_config_t", "ServeConfig"),
                                          ("mpx_serve_result_t", "ServeResult"),
                                          ("mpx_world_config_t", "WorldConfig"),
                                          ("mpx_status_t", "Status"),
                                          ("mpx_hostrate_config_t", "HostrateConfig"),
                                          ("mpx_hostrate_result_t", "HostrateResult"),
                                          ("mpx_serve_schedule_t", "ServeSchedule")])
def test_struct_layouts_match_the_binding(tmp_path, cname, pyname):
    import subprocess
    from paper_2208_13707_gb300 import mpx
    cls = getattr(mpx, pyname)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / "l.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mpx.h"\nint main(void){\n'
                   f'  printf("%zu", sizeof({cname}));\n' +
                   "".join(f'  printf(" %zu", offsetof({cname}, {f}));\n' for f in fields) +
                   "  return 0;\n}\n")
    exe = tmp_path / "l"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(cls)
    assert out[1:] == [getattr(cls, f).offset for f in fields]


def test_serve_run_rejects_bad_configs_without_a_gpu():
    from paper_2208_13707_gb300 import mpx
    c = mpx.mpx_serve_config_init()
    assert c.nthreads == 32 and c.max_log2 == 24 and abs(c.p_allreduce - 0.3) < 1e-12
    c.nthreads = 1
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_serve_run(c)
    assert e.value.code == mpx.ERR_ARG


def _header_constants():
    """Every enum constant of include/mpx.h (MPX_ prefix, upper case)."""
    src = open(os.path.join(ROOT, "include", "mpx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = []
    for body in re.findall(r"\benum\s*\{(.*?)\}", src, flags=re.S):
        for item in body.split(","):
            m = re.match(r"\s*(MPX_[A-Z0-9_]+)\b", item)
            if m:
                names.append(m.group(1))
    return names


def test_constants_match_the_binding(tmp_path):
    """Each MPX_* constant as the C compiler evaluates it equals the binding's
    value of the same name without the prefix, and the traffic program format
    uses the header's wildcard and status error values."""
    import subprocess
    from paper_2208_13707_gb300 import mpx
    from traffic import program
    names = _header_constants()
    assert len(names) > 60
    macros = ["MPX_REQUEST_NULL"]
    src = tmp_path / "c.c"
    src.write_text('#include <stdio.h>\n#include "mpx.h"\nint main(void){\n' +
                   "".join(f'  printf("{n} %lld\\n", (long long)({n}));\n' for n in names + macros) +
                   '  printf("MPX_IN_PLACE %lld\\n", (long long)(size_t)MPX_IN_PLACE);\n'
                   "  return 0;\n}\n")
    exe = tmp_path / "c"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    wrong = [(n, int(v), getattr(mpx, n[4:], None)) for n, v in got.items()
             if getattr(mpx, n[4:], None) != int(v)]
    assert wrong == [], "binding constants that differ from include/mpx.h (name, C, Python)"
    assert (program.ANY_SOURCE, program.ANY_TAG, program.ANY_INDEX) == (
        int(got["MPX_ANY_SOURCE"]), int(got["MPX_ANY_TAG"]), int(got["MPX_ANY_INDEX"]))
    assert (program.ERR_TRUNCATE, program.ERR_TIMEOUT) == (
        int(got["MPX_ERR_TRUNCATE"]), int(got["MPX_ERR_TIMEOUT"]))
    assert [program.T_BYTE, program.T_INT32, program.T_INT64, program.T_FLOAT, program.T_DOUBLE] == [
        int(got[n]) for n in ("MPX_BYTE", "MPX_INT32", "MPX_INT64", "MPX_FLOAT", "MPX_DOUBLE")]


_NULL_CALLS = r'''
import ctypes, sys
lib = ctypes.CDLL(sys.argv[1])
for item in sys.argv[2:]:
    name, nargs = item.split(":")
    f = getattr(lib, name)
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * int(nargs)
    print(name, end=" ", flush=True)
    print(f(*([None] * int(nargs))), flush=True)
'''


def test_null_handles_and_zero_sizes_return_codes(lib):
    """Every entry point called with null pointers, null handles and zero
    sizes returns an error code without crashing and without touching a GPU;
    only calls that a zero count makes no-ops (waitall and startall of no
    requests, an empty batch, an axpy of no elements, a zero-byte static
    copy) succeed.  One child process makes every call in turn, so a crash
    names the call."""
    import subprocess
    import sys
    src = open(os.path.join(ROOT, "include", "mpx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = re.findall(r"\bint\s+(mpx_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", src)
    assert len(decls) == len(_declared())
    items = [f"{n}:{0 if a.strip() in ('', 'void') else len(a.split(','))}" for n, a in decls]
    path = os.path.join(ROOT, "paper_2208_13707_gb300", "_lib", "libmpx.so")
    r = subprocess.run([sys.executable, "-c", _NULL_CALLS, path, *items], capture_output=True,
                       text=True, timeout=300, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    lines = r.stdout.splitlines()
    assert r.returncode == 0, f"crashed in {lines[-1] if lines else '?'}: {r.stderr[-300:]}"
    got = dict(line.split() for line in lines)
    assert len(got) == len(decls)
    no_ops = {"mpx_waitall_enqueue", "mpx_startall_enqueue", "mpx_enqueue_batch",
              "mpx_saxpy_enqueue", "mpx_sendrecv_static", "mpx_version"}
    ok = sorted(n for n, v in got.items() if int(v) == 0)
    assert set(ok) <= no_ops, f"calls that succeed on null arguments: {sorted(set(ok) - no_ops)}"


def test_datatype_registry_from_many_threads():
    """Derived datatypes are process-wide: threads that create, check and free
    vector types at the same time get distinct live handles whose size and
    extent are their own (ctypes releases the interpreter lock during each
    call, so the calls overlap in the library)."""
    import threading
    from paper_2208_13707_gb300 import mpx
    errors, live = [], {}
    lock = threading.Lock()

    def worker(t):
        try:
            for k in range(300):
                vc, bl = 1 + (t + k) % 7, 1 + k % 5
                st = bl + t % 3
                h = mpx.mpx_type_vector(vc, bl, st, mpx.INT32)
                with lock:
                    if h in live:
                        errors.append(f"handle {h} handed out twice")
                    live[h] = t
                if mpx.mpx_type_size(h) != 4 * vc * bl or \
                        mpx.mpx_type_extent(h) != 4 * ((vc - 1) * st + bl):
                    errors.append(f"type {h} of thread {t} changed")
                with lock:
                    del live[h]
                mpx.mpx_type_free(h)
        except Exception as e:      # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(8)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert errors == []


_CONFIG_FIELDS = {   # field: (environment variable, default documented in include/mpx.h)
    "engine_mode": ("MPX_ENGINE_MODE", 0), "max_streams": ("MPX_MAX_STREAMS", 64),
    "ring_slots": ("MPX_RING_SLOTS", 4096), "max_comms": ("MPX_MAX_COMMS", 8),
    "queue_slots": ("MPX_QUEUE_SLOTS", 4096), "task_slots": ("MPX_TASK_SLOTS", 16384),
    "engine_ctas": ("MPX_ENGINE_CTAS", 0), "engine_threads": ("MPX_ENGINE_THREADS", 256),
    "tile_bytes": ("MPX_TILE_BYTES", 65536), "bulk_min_bytes": ("MPX_BULK_MIN_BYTES", 32768),
    "reduce_mode": ("MPX_REDUCE_MODE", 0), "mover_schedule": ("MPX_MOVER_SCHEDULE", 0),
    "staging_bytes": ("MPX_STAGING_BYTES", 256 << 20), "budget_bytes": ("MPX_BUDGET_BYTES", 0),
    "watchdog_ns": ("MPX_WATCHDOG_NS", 10 ** 10), "idle_exit_ns": ("MPX_IDLE_EXIT_NS", 10 ** 8),
    "stage_delay_ns": ("MPX_STAGE_DELAY_NS", 20000), "ring_placement": ("MPX_RING_PLACEMENT", 0),
}

_CONFIG_DUMP = r'''
import json, sys
sys.path.insert(0, sys.argv[1])
from paper_2208_13707_gb300 import mpx
c = mpx.mpx_world_config_init()
print(json.dumps({f: getattr(c, f) for f, _ in c._fields_}))
'''


def _config_in_env(env_over):
    import json
    import subprocess
    import sys
    env = {k: v for k, v in os.environ.items() if not k.startswith("MPX_")}
    env.update(env_over)
    r = subprocess.run([sys.executable, "-c", _CONFIG_DUMP, ROOT], capture_output=True, text=True,
                       env=env, timeout=120, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_config_defaults_are_the_documented_ones_and_env_overrides_each_field():
    got = _config_in_env({})
    assert {f: got[f] for f in _CONFIG_FIELDS} == {f: d for f, (_, d) in _CONFIG_FIELDS.items()}
    over = {env: str(d + 1 if d else 7) for f, (env, d) in _CONFIG_FIELDS.items()}
    got = _config_in_env(over)
    assert {f: got[f] for f in _CONFIG_FIELDS} == {f: int(over[env]) for f, (env, _) in _CONFIG_FIELDS.items()}


@pytest.mark.parametrize("field,value", [
    ("max_streams", 0), ("max_streams", 1025), ("ring_slots", 8), ("queue_slots", 48),
    ("queue_slots", 16), ("task_slots", 32), ("max_comms", 0), ("max_comms", 65536),
    ("tile_bytes", 128), ("tile_bytes", 4100), ("engine_threads", 32), ("engine_threads", 544),
    ("engine_threads", 100), ("engine_mode", 3), ("engine_mode", -1), ("staging_bytes", 4095),
    ("mover_schedule", 2), ("ring_placement", -1)])
def test_world_config_out_of_range_is_refused_before_any_cuda_call(field, value):
    from paper_2208_13707_gb300 import mpx
    cfg = mpx.mpx_world_config_init()
    setattr(cfg, field, value)
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_world_create(2, cfg)
    assert e.value.code == mpx.ERR_ARG
    for n in (0, 4097):
        with pytest.raises(mpx.MpxError) as e:
            mpx.mpx_world_create(n, None)
        assert e.value.code == mpx.ERR_ARG
