"""ctypes binding of libmpx.so (include/mpx.h): same names, argument
marshalling only.  Every call that returns an error code raises MpxError with
that code (`.code`); `lib` gives the raw functions.  Raises at import time
when the library has not been built: there is no fallback path."""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmpx.so")

# see include/mpx.h: unsatisfied stream waits stall their hardware queue
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libmpx.so is not built ({LIB_PATH}); run paper_2208_13707_gb300.build.build()")

lib = ctypes.CDLL(LIB_PATH, mode=ctypes.RTLD_GLOBAL)

# --- constants (include/mpx.h) ---
ANY_SOURCE, ANY_TAG, TAG_UB, UNDEFINED = -2, -1, (1 << 30) - 1, -32766
ANY_INDEX = -1
MAX_INFO_KEY, MAX_INFO_VAL = 255, 1024
BYTE = UINT8 = 0
INT32, INT64, FLOAT, DOUBLE = 1, 2, 3, 4
SUM = 0
REDUCE_FIXED, REDUCE_TREE = 0, 1
STREAM_DEFAULT, STREAM_EXCLUSIVE = 0, 1
ENGINE_PERSISTENT, ENGINE_DRAIN, ENGINE_PLAIN = 0, 1, 2
MOVERS_WORKLIST, MOVERS_PER_CTA = 0, 1
RINGS_HOST, RINGS_DEVICE = 0, 1
REQUEST_NULL = -1
IN_PLACE = 1
ERRORS = {0: "SUCCESS", 1: "ERR_ARG", 2: "ERR_RANK", 3: "ERR_TAG", 4: "ERR_TYPE", 5: "ERR_COMM",
          6: "ERR_NO_ENDPOINT", 7: "ERR_AGAIN", 8: "ERR_STREAM", 9: "ERR_PENDING", 10: "ERR_CUDA",
          11: "ERR_REQUEST", 12: "ERR_NO_MEM", 13: "ERR_STATE", 14: "ERR_INTERN",
          15: "ERR_TRUNCATE", 16: "ERR_TIMEOUT", 17: "ERR_UNSUPPORTED"}
globals().update({"ERR_" + v[4:] if v.startswith("ERR_") else v: k for k, v in ERRORS.items()})


class MpxError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        super().__init__(f"{where}: MPX_{ERRORS.get(code, code)}")
        self.code = code


class WorldConfig(ctypes.Structure):
    _fields_ = [("engine_mode", ctypes.c_int32), ("max_streams", ctypes.c_int32),
                ("ring_slots", ctypes.c_int32), ("max_comms", ctypes.c_int32),
                ("queue_slots", ctypes.c_int32), ("task_slots", ctypes.c_int32),
                ("engine_ctas", ctypes.c_int32), ("engine_threads", ctypes.c_int32),
                ("tile_bytes", ctypes.c_int32), ("bulk_min_bytes", ctypes.c_int32),
                ("reduce_mode", ctypes.c_int32), ("mover_schedule", ctypes.c_int32),
                ("staging_bytes", ctypes.c_int64), ("budget_bytes", ctypes.c_int64),
                ("watchdog_ns", ctypes.c_int64), ("idle_exit_ns", ctypes.c_int64),
                ("stage_delay_ns", ctypes.c_int64), ("ring_placement", ctypes.c_int32),
                ("reserved0", ctypes.c_int32)]


(OP_SEND, OP_RECV, OP_ISEND, OP_IRECV, OP_WAIT, OP_WAITALL, OP_ALLREDUCE, OP_BCAST, OP_REDUCE,
 OP_ALLGATHER, OP_BARRIER) = range(11)


def op_dtype():
    """numpy layout of mpx_op_t (72 bytes), for building batches as arrays."""
    import numpy as np
    return np.dtype([("kind", "<i4"), ("datatype", "<i4"), ("peer", "<i4"), ("tag", "<i4"),
                     ("count", "<i8"), ("buf", "<u8"), ("recvbuf", "<u8"), ("comm", "<u8"),
                     ("requests", "<u8"), ("status", "<u8"), ("op", "<i4"), ("pad", "<i4")])


class ServeConfig(ctypes.Structure):
    _fields_ = [("nthreads", ctypes.c_int32), ("engine_mode", ctypes.c_int32),
                ("requests", ctypes.c_int64), ("mean_gap_us", ctypes.c_double),
                ("zipf_s", ctypes.c_double), ("min_log2", ctypes.c_int32), ("max_log2", ctypes.c_int32),
                ("p_allreduce", ctypes.c_double), ("budget_bytes", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("sample_every", ctypes.c_int64), ("only_item", ctypes.c_int64)]


class ServeResult(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("items", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("msgs_per_s", ctypes.c_double), ("gbs", ctypes.c_double),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("svc_p50_us", ctypes.c_double), ("svc_p99_us", ctypes.c_double),
                ("admission_waits", ctypes.c_int64), ("peak_bytes", ctypes.c_int64)]


SERVE_SEND, SERVE_RECV, SERVE_WAITALL, SERVE_ALLREDUCE = 0, 1, 2, 3


def serve_call_dtype():
    """numpy layout of mpx_serve_call_t."""
    import numpy as np
    return np.dtype([("kind", "<i4"), ("peer", "<i4"), ("tag", "<i4"), ("pad", "<i4"),
                     ("item", "<i8"), ("bytes", "<i8"), ("off", "<i8"), ("capture", "<i8")])


class ServeSchedule(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_void_p), ("call_lo", ctypes.c_void_p), ("regions", ctypes.c_void_p),
                ("region_bytes", ctypes.c_int64), ("capture", ctypes.c_void_p),
                ("capture_bytes", ctypes.c_int64), ("statuses", ctypes.c_void_p),
                ("nstatuses", ctypes.c_int64)]


class Status(ctypes.Structure):
    _fields_ = [("source", ctypes.c_int32), ("tag", ctypes.c_int32), ("error", ctypes.c_int32),
                ("source_index", ctypes.c_int32), ("bytes", ctypes.c_int64)]


HOSTRATE_GLOBAL_LOCK, HOSTRATE_ENDPOINT_LOCK, HOSTRATE_STREAM = 0, 1, 2


class HostrateConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("mode", ctypes.c_int32), ("messages", ctypes.c_int64),
                ("window", ctypes.c_int32), ("pad", ctypes.c_int32)]


class HostrateResult(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("msgs_per_s", ctypes.c_double),
                ("errors", ctypes.c_int64)]


_vp, _i32, _i64, _u32, _f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float
_P = ctypes.POINTER
_SIGS = {
    "mpx_world_config_init": [_P(WorldConfig)],
    "mpx_world_create": [ctypes.c_int, _P(WorldConfig), _P(_vp)],
    "mpx_world_free": [_P(_vp)],
    "mpx_world_start": [_vp],
    "mpx_world_stop": [_vp, ctypes.c_int],
    "mpx_world_progress": [_vp, _vp],
    "mpx_world_abort": [_vp],
    "mpx_world_debug_dump": [_vp],
    "mpx_world_get_error": [_vp, _P(ctypes.c_int)],
    "mpx_world_get_counters": [_vp, _P(_i64), ctypes.c_int],
    "mpx_stream_create": [_vp, ctypes.c_int, _vp, ctypes.c_uint, _P(_vp)],
    "mpx_stream_free": [_P(_vp)],
    "mpx_stream_get_id": [_vp, _P(ctypes.c_int)],
    "mpx_stream_get_error": [_vp, _P(ctypes.c_int)],
    "mpx_stream_pending": [_vp, _P(_i64)],
    "mpx_hostrate_config_init": [_P(HostrateConfig)],
    "mpx_hostrate_run": [_P(HostrateConfig), _P(HostrateResult)],
    "mpx_stream_create_info": [_vp, ctypes.c_int, _vp, _P(_vp)],
    "mpx_stream_get_cuda_stream": [_vp, _P(_vp)],
    "mpx_info_create": [_P(_vp)],
    "mpx_info_free": [_P(_vp)],
    "mpx_info_set": [_vp, ctypes.c_char_p, ctypes.c_char_p],
    "mpx_info_get": [_vp, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, _P(ctypes.c_int)],
    "mpx_info_get_valuelen": [_vp, ctypes.c_char_p, _P(ctypes.c_int), _P(ctypes.c_int)],
    "mpx_info_get_nkeys": [_vp, _P(ctypes.c_int)],
    "mpx_info_get_nthkey": [_vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_int],
    "mpx_info_set_hex": [_vp, ctypes.c_char_p, _vp, ctypes.c_int],
    "mpx_info_get_hex": [_vp, ctypes.c_char_p, _vp, ctypes.c_int, _P(ctypes.c_int)],
    "mpx_stream_comm_create": [_vp, ctypes.c_int, _P(_vp), _P(_vp)],
    "mpx_stream_comm_create_multiple": [_vp, ctypes.c_int, _P(ctypes.c_int), _P(_vp), _P(_vp)],
    "mpx_comm_free": [_P(_vp)],
    "mpx_comm_rank": [_vp, _P(ctypes.c_int)],
    "mpx_comm_size": [_vp, _P(ctypes.c_int)],
    "mpx_comm_set_reduce_mode": [_vp, ctypes.c_int],
    "mpx_type_vector": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32, _P(_i32)],
    "mpx_type_free": [_P(_i32)],
    "mpx_type_size": [_i32, _P(_i64)],
    "mpx_type_extent": [_i32, _P(_i64)],
    "mpx_send_enqueue": [_vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp],
    "mpx_recv_enqueue": [_vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp, _vp],
    "mpx_isend_enqueue": [_vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp, _P(_i64)],
    "mpx_irecv_enqueue": [_vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp, _P(_i64)],
    "mpx_stream_send_enqueue": [_vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int,
                                ctypes.c_int],
    "mpx_stream_recv_enqueue": [_vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int,
                                ctypes.c_int, _vp],
    "mpx_stream_isend_enqueue": [_vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int,
                                 ctypes.c_int, _P(_i64)],
    "mpx_stream_irecv_enqueue": [_vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int,
                                 ctypes.c_int, _P(_i64)],
    "mpx_wait_enqueue": [_P(_i64), _vp],
    "mpx_waitall_enqueue": [ctypes.c_int, _P(_i64), _vp],
    "mpx_allreduce_enqueue": [_vp, _vp, _i64, _i32, ctypes.c_int, _vp],
    "mpx_bcast_enqueue": [_vp, _i64, _i32, ctypes.c_int, _vp],
    "mpx_reduce_enqueue": [_vp, _vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp],
    "mpx_allgather_enqueue": [_vp, _vp, _i64, _i32, _vp],
    "mpx_barrier_enqueue": [_vp],
    "mpx_iallreduce_enqueue": [_vp, _vp, _i64, _i32, ctypes.c_int, _vp, _P(_i64)],
    "mpx_ibcast_enqueue": [_vp, _i64, _i32, ctypes.c_int, _vp, _P(_i64)],
    "mpx_ireduce_enqueue": [_vp, _vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp, _P(_i64)],
    "mpx_iallgather_enqueue": [_vp, _vp, _i64, _i32, _vp, _P(_i64)],
    "mpx_ibarrier_enqueue": [_vp, _P(_i64)],
    "mpx_allreduce_init": [_vp, _vp, _i64, _i32, ctypes.c_int, _vp, _P(_i64)],
    "mpx_bcast_init": [_vp, _i64, _i32, ctypes.c_int, _vp, _P(_i64)],
    "mpx_reduce_init": [_vp, _vp, _i64, _i32, ctypes.c_int, ctypes.c_int, _vp, _P(_i64)],
    "mpx_allgather_init": [_vp, _vp, _i64, _i32, _vp, _P(_i64)],
    "mpx_barrier_init": [_vp, _P(_i64)],
    "mpx_start_enqueue": [_P(_i64)],
    "mpx_startall_enqueue": [ctypes.c_int, _P(_i64)],
    "mpx_request_free": [_P(_i64)],
    "mpx_get_count": [_P(Status), _i32, _P(_i64)],
    "mpx_saxpy_enqueue": [_i64, _f32, _vp, _vp, _vp],
    "mpx_sendrecv_static": [_vp, _i64, _i32, _vp, _i64, _i32, _vp, _P(_i64)],
    "mpx_enqueue_batch": [ctypes.c_int, _vp, _P(ctypes.c_int)],
    "mpx_step_create": [_vp, ctypes.c_int, _vp, _P(_vp)],
    "mpx_serve_config_init": [_P(ServeConfig)],
    "mpx_serve_run": [_P(ServeConfig), _P(ServeResult), _vp, _vp, _i64],
    "mpx_serve_run_schedule": [_P(ServeConfig), _P(ServeSchedule), _P(ServeResult)],
    "mpx_step_launch": [_vp, _vp],
    "mpx_step_get_error": [_vp, _P(ctypes.c_int)],
    "mpx_step_free": [_P(_vp)],
    "mpx_version": [],
    "mpx_cuda_stream_create": [_P(_vp)],
    "mpx_cuda_stream_destroy": [_vp],
}
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int


def _chk(rc: int, where: str):
    if rc != 0:
        raise MpxError(rc, where)


# --- world ---
def mpx_world_config_init() -> WorldConfig:
    c = WorldConfig()
    _chk(lib.mpx_world_config_init(ctypes.byref(c)), "mpx_world_config_init")
    return c


def mpx_world_create(nranks: int, cfg: Optional[WorldConfig] = None) -> int:
    w = _vp()
    _chk(lib.mpx_world_create(nranks, ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(w)),
         "mpx_world_create")
    return w.value


def mpx_world_free(world: int) -> None:
    w = _vp(world)
    _chk(lib.mpx_world_free(ctypes.byref(w)), "mpx_world_free")


def mpx_world_start(world: int) -> None:
    _chk(lib.mpx_world_start(world), "mpx_world_start")


def mpx_world_stop(world: int, timeout_ms: int = 10000) -> None:
    _chk(lib.mpx_world_stop(world, timeout_ms), "mpx_world_stop")


def mpx_world_progress(world: int, stream: int) -> None:
    _chk(lib.mpx_world_progress(world, stream), "mpx_world_progress")


def mpx_world_abort(world: int) -> None:
    _chk(lib.mpx_world_abort(world), "mpx_world_abort")


def mpx_world_debug_dump(world: int) -> None:
    lib.mpx_world_debug_dump(world)


def mpx_world_get_error(world: int) -> int:
    e = ctypes.c_int()
    _chk(lib.mpx_world_get_error(world, ctypes.byref(e)), "mpx_world_get_error")
    return e.value


def mpx_world_get_counters(world: int) -> list:
    a = (_i64 * 27)()
    _chk(lib.mpx_world_get_counters(world, a, 27), "mpx_world_get_counters")
    return list(a)


lib.mpxi_world_trace.argtypes = [_vp, _vp, _i64]
lib.mpxi_world_trace.restype = _i64
lib.mpxi_device_attr.argtypes = [ctypes.c_int, _P(ctypes.c_int)]
lib.mpxi_device_attr.restype = ctypes.c_int


def device_attr(attr: int) -> int:
    """Diagnostic: cudaDeviceGetAttribute(attr) of the current device."""
    v = ctypes.c_int()
    _chk(lib.mpxi_device_attr(attr, ctypes.byref(v)), "mpxi_device_attr")
    return v.value


def engine_trace(world: int, max_records: int = 1 << 16):
    """Diagnostic: the engine's timeline records since the last call, as a
    (k, 4) uint64 array, and restart the trace.  Needs the environment variable
    MPX_ENGINE_TRACE (record capacity) set before the world is created; empty
    otherwise.  A mover tile writes (start ns, end ns, task << 32 | tile,
    bytes << 8 | kind bits); a control tick writes (start ns, end ns,
    0xFFFFFFFF << 32 | tick, what it did: bit 0 ingest, bit 1 new events,
    bit 2 completion scan, bits 8-31 tasks outstanding, bits 32+ tasks made)
    and then (start ns, four 16-bit phase ends, 0xFFFFFFFE << 32 | tick, four
    more): microseconds from the tick's start at the ends of ingest, rounds,
    finished tasks, completion, scheduling scans, listed receives, deferred
    deliveries and scheduling (0: phase not reached)."""
    import numpy as np
    out = np.zeros((max_records, 4), np.uint64)
    k = lib.mpxi_world_trace(world, out.ctypes.data, max_records)
    if k < 0:
        raise MpxError(ERR_CUDA, "mpxi_world_trace")
    return out[:k]


# --- streams and communicators ---
def mpx_stream_create(world: int, rank: int, cuda_stream: int, flags: int = 0) -> int:
    s = _vp()
    _chk(lib.mpx_stream_create(world, rank, cuda_stream, flags, ctypes.byref(s)), "mpx_stream_create")
    return s.value


def mpx_stream_free(stream: int) -> None:
    s = _vp(stream)
    _chk(lib.mpx_stream_free(ctypes.byref(s)), "mpx_stream_free")


def mpx_stream_get_id(stream: int) -> int:
    i = ctypes.c_int()
    _chk(lib.mpx_stream_get_id(stream, ctypes.byref(i)), "mpx_stream_get_id")
    return i.value


def mpx_stream_get_error(stream: int) -> int:
    e = ctypes.c_int()
    _chk(lib.mpx_stream_get_error(stream, ctypes.byref(e)), "mpx_stream_get_error")
    return e.value


def mpx_stream_pending(stream: int) -> int:
    n = _i64()
    _chk(lib.mpx_stream_pending(stream, ctypes.byref(n)), "mpx_stream_pending")
    return n.value


def mpx_stream_comm_create(world: int, streams: Sequence[int]) -> list:
    n = len(streams)
    arr = (_vp * n)(*streams)
    out = (_vp * n)()
    _chk(lib.mpx_stream_comm_create(world, n, arr, out), "mpx_stream_comm_create")
    return [out[i] for i in range(n)]


def mpx_hostrate_config_init() -> HostrateConfig:
    cfg = HostrateConfig()
    _chk(lib.mpx_hostrate_config_init(ctypes.byref(cfg)), "mpx_hostrate_config_init")
    return cfg


def mpx_hostrate_run(threads: int, mode: int, messages: int = 1 << 20, window: int = 64) -> dict:
    """Host-thread 8-byte message rate under one locking discipline (HOSTRATE_*)."""
    cfg = mpx_hostrate_config_init()
    cfg.threads, cfg.mode, cfg.messages, cfg.window = threads, mode, messages, window
    res = HostrateResult()
    _chk(lib.mpx_hostrate_run(ctypes.byref(cfg), ctypes.byref(res)), "mpx_hostrate_run")
    return {"seconds": res.seconds, "msgs_per_s": res.msgs_per_s, "errors": int(res.errors)}


def mpx_stream_create_info(world: int, rank: int, info: Optional[int]) -> int:
    """MPIX_Stream_create from info hints; info None = MPI_INFO_NULL."""
    out = _vp()
    _chk(lib.mpx_stream_create_info(world, rank, info, ctypes.byref(out)), "mpx_stream_create_info")
    return out.value


def mpx_stream_get_cuda_stream(stream: int) -> int:
    out = _vp()
    _chk(lib.mpx_stream_get_cuda_stream(stream, ctypes.byref(out)), "mpx_stream_get_cuda_stream")
    return out.value or 0


def mpx_info_create() -> int:
    out = _vp()
    _chk(lib.mpx_info_create(ctypes.byref(out)), "mpx_info_create")
    return out.value


def mpx_info_free(info: int) -> None:
    h = _vp(info)
    _chk(lib.mpx_info_free(ctypes.byref(h)), "mpx_info_free")


def mpx_info_set(info: int, key: str, value: str) -> None:
    _chk(lib.mpx_info_set(info, key.encode(), value.encode()), "mpx_info_set")


def mpx_info_get(info: int, key: str, buflen: int = MAX_INFO_VAL + 1) -> Optional[str]:
    buf = ctypes.create_string_buffer(max(1, buflen))
    flag = ctypes.c_int()
    _chk(lib.mpx_info_get(info, key.encode(), buf, buflen, ctypes.byref(flag)), "mpx_info_get")
    return buf.value.decode() if flag.value else None


def mpx_info_get_valuelen(info: int, key: str) -> Optional[int]:
    n, flag = ctypes.c_int(), ctypes.c_int()
    _chk(lib.mpx_info_get_valuelen(info, key.encode(), ctypes.byref(n), ctypes.byref(flag)),
         "mpx_info_get_valuelen")
    return n.value if flag.value else None


def mpx_info_get_nkeys(info: int) -> int:
    n = ctypes.c_int()
    _chk(lib.mpx_info_get_nkeys(info, ctypes.byref(n)), "mpx_info_get_nkeys")
    return n.value


def mpx_info_get_nthkey(info: int, n: int) -> str:
    buf = ctypes.create_string_buffer(MAX_INFO_KEY + 1)
    _chk(lib.mpx_info_get_nthkey(info, n, buf, MAX_INFO_KEY + 1), "mpx_info_get_nthkey")
    return buf.value.decode()


def mpx_info_set_hex(info: int, key: str, value: bytes) -> None:
    """MPIX_Info_set_hex: store the bytes of `value` under `key`."""
    b = ctypes.create_string_buffer(bytes(value), len(value))
    _chk(lib.mpx_info_set_hex(info, key.encode(), b, len(value)), "mpx_info_set_hex")


def mpx_info_get_hex(info: int, key: str, vallen: int) -> Optional[bytes]:
    b = ctypes.create_string_buffer(max(1, vallen))
    flag = ctypes.c_int()
    _chk(lib.mpx_info_get_hex(info, key.encode(), b, vallen, ctypes.byref(flag)), "mpx_info_get_hex")
    return b.raw[:vallen] if flag.value else None


def mpx_stream_comm_create_multiple(world: int, local_streams: Sequence[Sequence[int]]) -> list:
    """local_streams[r]: rank r's streams in local-index order; returns one handle per rank."""
    n = len(local_streams)
    counts = (ctypes.c_int * n)(*[len(l) for l in local_streams])
    flat = [h for l in local_streams for h in l]
    arr = (_vp * max(1, len(flat)))(*flat)
    out = (_vp * n)()
    _chk(lib.mpx_stream_comm_create_multiple(world, n, counts, arr, out),
         "mpx_stream_comm_create_multiple")
    return [out[i] for i in range(n)]


def mpx_comm_free(comm: int) -> None:
    c = _vp(comm)
    _chk(lib.mpx_comm_free(ctypes.byref(c)), "mpx_comm_free")


def mpx_comm_rank(comm: int) -> int:
    r = ctypes.c_int()
    _chk(lib.mpx_comm_rank(comm, ctypes.byref(r)), "mpx_comm_rank")
    return r.value


def mpx_comm_size(comm: int) -> int:
    r = ctypes.c_int()
    _chk(lib.mpx_comm_size(comm, ctypes.byref(r)), "mpx_comm_size")
    return r.value


def mpx_comm_set_reduce_mode(comm: int, mode: int) -> None:
    _chk(lib.mpx_comm_set_reduce_mode(comm, mode), "mpx_comm_set_reduce_mode")


# --- datatypes ---
def mpx_type_vector(count: int, blocklength: int, stride: int, oldtype: int) -> int:
    t = _i32()
    _chk(lib.mpx_type_vector(count, blocklength, stride, oldtype, ctypes.byref(t)), "mpx_type_vector")
    return t.value


def mpx_type_free(t: int) -> None:
    x = _i32(t)
    _chk(lib.mpx_type_free(ctypes.byref(x)), "mpx_type_free")


def mpx_type_size(t: int) -> int:
    x = _i64()
    _chk(lib.mpx_type_size(t, ctypes.byref(x)), "mpx_type_size")
    return x.value


def mpx_type_extent(t: int) -> int:
    x = _i64()
    _chk(lib.mpx_type_extent(t, ctypes.byref(x)), "mpx_type_extent")
    return x.value


# --- enqueue (buffers and statuses are device addresses as ints) ---
def mpx_send_enqueue(buf: int, count: int, datatype: int, dest: int, tag: int, comm: int) -> None:
    _chk(lib.mpx_send_enqueue(buf, count, datatype, dest, tag, comm), "mpx_send_enqueue")


def mpx_recv_enqueue(buf: int, count: int, datatype: int, source: int, tag: int, comm: int,
                     status: int = 0) -> None:
    _chk(lib.mpx_recv_enqueue(buf, count, datatype, source, tag, comm, status or None), "mpx_recv_enqueue")


def mpx_isend_enqueue(buf: int, count: int, datatype: int, dest: int, tag: int, comm: int) -> int:
    r = _i64()
    _chk(lib.mpx_isend_enqueue(buf, count, datatype, dest, tag, comm, ctypes.byref(r)), "mpx_isend_enqueue")
    return r.value


def mpx_irecv_enqueue(buf: int, count: int, datatype: int, source: int, tag: int, comm: int) -> int:
    r = _i64()
    _chk(lib.mpx_irecv_enqueue(buf, count, datatype, source, tag, comm, ctypes.byref(r)), "mpx_irecv_enqueue")
    return r.value


def mpx_stream_send_enqueue(buf: int, count: int, datatype: int, dest: int, tag: int, comm: int,
                            src_idx: int, dst_idx: int) -> None:
    _chk(lib.mpx_stream_send_enqueue(buf, count, datatype, dest, tag, comm, src_idx, dst_idx),
         "mpx_stream_send_enqueue")


def mpx_stream_recv_enqueue(buf: int, count: int, datatype: int, source: int, tag: int, comm: int,
                            src_idx: int, dst_idx: int, status: int = 0) -> None:
    _chk(lib.mpx_stream_recv_enqueue(buf, count, datatype, source, tag, comm, src_idx, dst_idx,
                                     status or None), "mpx_stream_recv_enqueue")


def mpx_stream_isend_enqueue(buf: int, count: int, datatype: int, dest: int, tag: int, comm: int,
                             src_idx: int, dst_idx: int) -> int:
    r = _i64()
    _chk(lib.mpx_stream_isend_enqueue(buf, count, datatype, dest, tag, comm, src_idx, dst_idx,
                                      ctypes.byref(r)), "mpx_stream_isend_enqueue")
    return r.value


def mpx_stream_irecv_enqueue(buf: int, count: int, datatype: int, source: int, tag: int, comm: int,
                             src_idx: int, dst_idx: int) -> int:
    r = _i64()
    _chk(lib.mpx_stream_irecv_enqueue(buf, count, datatype, source, tag, comm, src_idx, dst_idx,
                                      ctypes.byref(r)), "mpx_stream_irecv_enqueue")
    return r.value


def mpx_wait_enqueue(request: int, status: int = 0) -> None:
    r = _i64(request)
    _chk(lib.mpx_wait_enqueue(ctypes.byref(r), status or None), "mpx_wait_enqueue")


def mpx_waitall_enqueue(requests: Sequence[int], statuses: int = 0) -> None:
    n = len(requests)
    arr = (_i64 * max(1, n))(*requests)
    _chk(lib.mpx_waitall_enqueue(n, arr, statuses or None), "mpx_waitall_enqueue")


def mpx_allreduce_enqueue(sendbuf: int, recvbuf: int, count: int, datatype: int, op: int, comm: int) -> None:
    _chk(lib.mpx_allreduce_enqueue(sendbuf, recvbuf, count, datatype, op, comm), "mpx_allreduce_enqueue")


def mpx_bcast_enqueue(buf: int, count: int, datatype: int, root: int, comm: int) -> None:
    _chk(lib.mpx_bcast_enqueue(buf, count, datatype, root, comm), "mpx_bcast_enqueue")


def mpx_reduce_enqueue(sendbuf: int, recvbuf: int, count: int, datatype: int, op: int, root: int,
                       comm: int) -> None:
    _chk(lib.mpx_reduce_enqueue(sendbuf, recvbuf, count, datatype, op, root, comm), "mpx_reduce_enqueue")


def mpx_allgather_enqueue(sendbuf: int, recvbuf: int, count: int, datatype: int, comm: int) -> None:
    _chk(lib.mpx_allgather_enqueue(sendbuf, recvbuf, count, datatype, comm), "mpx_allgather_enqueue")


def mpx_barrier_enqueue(comm: int) -> None:
    _chk(lib.mpx_barrier_enqueue(comm), "mpx_barrier_enqueue")


def mpx_iallreduce_enqueue(sendbuf: int, recvbuf: int, count: int, datatype: int, op: int,
                           comm: int) -> int:
    r = _i64()
    _chk(lib.mpx_iallreduce_enqueue(sendbuf, recvbuf, count, datatype, op, comm, ctypes.byref(r)),
         "mpx_iallreduce_enqueue")
    return r.value


def mpx_ibcast_enqueue(buf: int, count: int, datatype: int, root: int, comm: int) -> int:
    r = _i64()
    _chk(lib.mpx_ibcast_enqueue(buf, count, datatype, root, comm, ctypes.byref(r)), "mpx_ibcast_enqueue")
    return r.value


def mpx_ireduce_enqueue(sendbuf: int, recvbuf: int, count: int, datatype: int, op: int, root: int,
                        comm: int) -> int:
    r = _i64()
    _chk(lib.mpx_ireduce_enqueue(sendbuf, recvbuf, count, datatype, op, root, comm, ctypes.byref(r)),
         "mpx_ireduce_enqueue")
    return r.value


def mpx_iallgather_enqueue(sendbuf: int, recvbuf: int, count: int, datatype: int, comm: int) -> int:
    r = _i64()
    _chk(lib.mpx_iallgather_enqueue(sendbuf, recvbuf, count, datatype, comm, ctypes.byref(r)),
         "mpx_iallgather_enqueue")
    return r.value


def mpx_ibarrier_enqueue(comm: int) -> int:
    r = _i64()
    _chk(lib.mpx_ibarrier_enqueue(comm, ctypes.byref(r)), "mpx_ibarrier_enqueue")
    return r.value


def mpx_get_count(status: Status, datatype: int) -> int:
    c = _i64()
    _chk(lib.mpx_get_count(ctypes.byref(status), datatype, ctypes.byref(c)), "mpx_get_count")
    return c.value


def mpx_saxpy_enqueue(n: int, a: float, x: int, y: int, stream: int) -> None:
    _chk(lib.mpx_saxpy_enqueue(n, a, x, y, stream), "mpx_saxpy_enqueue")


def mpx_cuda_stream_create() -> int:
    s = _vp()
    _chk(lib.mpx_cuda_stream_create(ctypes.byref(s)), "mpx_cuda_stream_create")
    return s.value


def mpx_cuda_stream_destroy(stream: int) -> None:
    _chk(lib.mpx_cuda_stream_destroy(stream), "mpx_cuda_stream_destroy")


def mpx_sendrecv_static(sendbuf: int, sendcount: int, sendtype: int, recvbuf: int, recvcount: int,
                        recvtype: int, stream: int) -> int:
    """Returns the number of bytes delivered."""
    n = _i64()
    _chk(lib.mpx_sendrecv_static(sendbuf, sendcount, sendtype, recvbuf, recvcount, recvtype, stream,
                                 ctypes.byref(n)), "mpx_sendrecv_static")
    return n.value


def mpx_version() -> int:
    return lib.mpx_version()


def mpx_enqueue_batch(ops, n: Optional[int] = None) -> int:
    """`ops`: a C-contiguous numpy array of op_dtype() (or anything exposing
    the buffer protocol with that layout).  Returns the number enqueued;
    raises MpxError (with `.done`) if an operation failed."""
    import numpy as np
    a = np.ascontiguousarray(ops)
    cnt = len(a) if n is None else int(n)
    done = ctypes.c_int(0)
    rc = lib.mpx_enqueue_batch(cnt, a.ctypes.data, ctypes.byref(done))
    if rc != 0:
        e = MpxError(rc, "mpx_enqueue_batch")
        e.done = done.value
        raise e
    return done.value


def mpx_step_create(world: int, ops) -> int:
    """Record the op_dtype() array `ops` as one step (see mpx_enqueue_batch for
    the layout); returns the step handle."""
    import numpy as np
    a = np.ascontiguousarray(ops)
    st = _vp()
    _chk(lib.mpx_step_create(world, len(a), a.ctypes.data, ctypes.byref(st)), "mpx_step_create")
    return st.value


def mpx_step_launch(step: int, stream: int) -> None:
    _chk(lib.mpx_step_launch(step, stream), "mpx_step_launch")


def mpx_step_get_error(step: int) -> int:
    e = ctypes.c_int(0)
    _chk(lib.mpx_step_get_error(step, ctypes.byref(e)), "mpx_step_get_error")
    return e.value


def mpx_step_free(step: int) -> None:
    st = _vp(step)
    _chk(lib.mpx_step_free(ctypes.byref(st)), "mpx_step_free")


def mpx_serve_config_init() -> ServeConfig:
    c = ServeConfig()
    _chk(lib.mpx_serve_config_init(ctypes.byref(c)), "mpx_serve_config_init")
    return c


def mpx_serve_run(cfg: ServeConfig, digests=None, source_digests=None) -> dict:
    """Run the serving loop; `digests` / `source_digests` (uint64 numpy arrays
    of one length, optional) receive the sampled items' digests as delivered
    and as sent.  Returns the result fields as a dict."""
    import numpy as np
    r = ServeResult()
    dp, sp, dn = (None, None, 0)
    if digests is not None:
        assert digests.dtype == np.uint64 and digests.flags.c_contiguous
        dp, dn = digests.ctypes.data, len(digests)
        if source_digests is not None:
            assert source_digests.dtype == np.uint64 and len(source_digests) == dn
            sp = source_digests.ctypes.data
    _chk(lib.mpx_serve_run(ctypes.byref(cfg), ctypes.byref(r), dp, sp, dn), "mpx_serve_run")
    return {k: getattr(r, k) for k, _ in ServeResult._fields_}


def mpx_serve_run_schedule(cfg: ServeConfig, calls, call_lo, regions, region_bytes: int,
                           capture: int = 0, capture_bytes: int = 0, statuses: int = 0,
                           nstatuses: int = 0) -> dict:
    """Run the serving loop over a caller-supplied schedule.  `calls` is a
    numpy array of serve_call_dtype(), `call_lo` int64 (nthreads + 1),
    `regions` a sequence of device pointers; capture / statuses are device
    pointers (0: none).  Returns the result fields as a dict."""
    import numpy as np
    calls = np.ascontiguousarray(calls, dtype=serve_call_dtype())
    call_lo = np.ascontiguousarray(call_lo, dtype=np.int64)
    regs = (ctypes.c_void_p * len(regions))(*[int(x) for x in regions])
    q = ServeSchedule(calls.ctypes.data, call_lo.ctypes.data, ctypes.cast(regs, ctypes.c_void_p),
                      int(region_bytes), capture or None, int(capture_bytes), statuses or None,
                      int(nstatuses))
    r = ServeResult()
    _chk(lib.mpx_serve_run_schedule(ctypes.byref(cfg), ctypes.byref(q), ctypes.byref(r)),
         "mpx_serve_run_schedule")
    return {k: getattr(r, k) for k, _ in ServeResult._fields_}


# --- persistent collectives ---------------------------------------------------
def _persist(fn, name, *args) -> int:
    r = _i64(-1)
    _chk(fn(*args, ctypes.byref(r)), name)
    return r.value


def mpx_allreduce_init(sendbuf: int, recvbuf: int, count: int, datatype: int, op: int, comm: int) -> int:
    return _persist(lib.mpx_allreduce_init, "mpx_allreduce_init", sendbuf, recvbuf, count, datatype, op, comm)


def mpx_bcast_init(buf: int, count: int, datatype: int, root: int, comm: int) -> int:
    return _persist(lib.mpx_bcast_init, "mpx_bcast_init", buf, count, datatype, root, comm)


def mpx_reduce_init(sendbuf: int, recvbuf: int, count: int, datatype: int, op: int, root: int,
                    comm: int) -> int:
    return _persist(lib.mpx_reduce_init, "mpx_reduce_init", sendbuf, recvbuf, count, datatype, op, root,
                    comm)


def mpx_allgather_init(sendbuf: int, recvbuf: int, count: int, datatype: int, comm: int) -> int:
    return _persist(lib.mpx_allgather_init, "mpx_allgather_init", sendbuf, recvbuf, count, datatype, comm)


def mpx_barrier_init(comm: int) -> int:
    return _persist(lib.mpx_barrier_init, "mpx_barrier_init", comm)


def mpx_start_enqueue(request: int) -> None:
    r = _i64(request)
    _chk(lib.mpx_start_enqueue(ctypes.byref(r)), "mpx_start_enqueue")


def mpx_startall_enqueue(requests) -> None:
    a = (_i64 * len(requests))(*requests)
    _chk(lib.mpx_startall_enqueue(len(requests), a), "mpx_startall_enqueue")


def mpx_request_free(request: int) -> None:
    r = _i64(request)
    _chk(lib.mpx_request_free(ctypes.byref(r)), "mpx_request_free")
