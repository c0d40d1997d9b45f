"""CPU oracle for enqueued MPI traffic programs (test infrastructure).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product library never links or calls
it.  `run(program)` executes a traffic program (see `traffic.program`) with the
single-threaded round model in `mpx_oracle.cpp` and returns the match map,
final buffer contents, statuses and per-op rounds.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpx_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CXXFLAGS = ["-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", *CXXFLAGS, "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Program(ctypes.Structure):
    _fields_ = [("nranks", ctypes.c_int32), ("nstreams", ctypes.c_int32),
                ("ncomms", ctypes.c_int32), ("ntypes", ctypes.c_int32),
                ("nops", ctypes.c_int64), ("nbufs", ctypes.c_int64),
                ("nreq", ctypes.c_int64), ("nstatus", ctypes.c_int64),
                ("stream_rank", ctypes.c_void_p), ("comm_stream", ctypes.c_void_p),
                ("stream_op_lo", ctypes.c_void_p), ("ops", ctypes.c_void_p),
                ("types", ctypes.c_void_p), ("bufs", ctypes.c_void_p),
                ("buf_size", ctypes.c_void_p), ("reqlist", ctypes.c_void_p),
                ("mux_off", ctypes.c_void_p), ("mux_stream", ctypes.c_void_p)]


class _Result(ctypes.Structure):
    _fields_ = [("match", ctypes.c_void_p), ("post_round", ctypes.c_void_p),
                ("done_round", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("stuck_op", ctypes.c_void_p), ("rounds", ctypes.c_int32),
                ("deadlock", ctypes.c_int32), ("error", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_run.argtypes = [ctypes.POINTER(_Program), ctypes.POINTER(_Result)]
            lib.oracle_run.restype = ctypes.c_int
            lib.oracle_sum_f32_ref.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_sum_f32_ref.restype = None
            _lib = lib
    return _lib


@dataclass
class OracleOutcome:
    buffers: List[np.ndarray]
    match: np.ndarray
    post_round: np.ndarray
    done_round: np.ndarray
    status: np.ndarray
    stuck_op: np.ndarray
    rounds: int
    deadlock: bool
    error: int


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def run(prog, buffers: Optional[List[np.ndarray]] = None) -> OracleOutcome:
    """Execute `prog` on CPU.  `buffers` (uint8 arrays, mutated) default to a
    fresh copy of the program's initial contents."""
    from traffic.program import STATUS_DTYPE  # format only
    lib = _load()
    bufs = prog.fresh_buffers() if buffers is None else buffers
    ops = np.ascontiguousarray(prog.ops)
    types = np.ascontiguousarray(prog.types)
    stream_rank = np.ascontiguousarray(prog.stream_rank, np.int32)
    comm_stream = np.ascontiguousarray(prog.comm_stream, np.int32)
    lo = np.ascontiguousarray(prog.stream_op_lo, np.int64)
    reqlist = np.ascontiguousarray(prog.reqlist, np.int64)
    ptrs = (ctypes.c_void_p * max(1, len(bufs)))(*[b.ctypes.data for b in bufs])
    sizes = np.array([b.size for b in bufs] or [0], np.int64)
    # multiplex comms: each rank's local streams, flattened (empty ranges elsewhere)
    mux_off = np.zeros(prog.ncomms * prog.nranks + 1, np.int64)
    mux_list: List[int] = []
    for c in range(prog.ncomms):
        m = prog.mux(c)
        for r in range(prog.nranks):
            if m is not None:
                mux_list.extend(int(g) for g in m[r])
            mux_off[c * prog.nranks + r + 1] = len(mux_list)
    mux_stream = np.array(mux_list or [0], np.int32)
    P = _Program(prog.nranks, prog.nstreams, prog.ncomms, len(types), len(ops), len(bufs),
                 len(reqlist), prog.nstatus, _ptr(stream_rank), _ptr(comm_stream), _ptr(lo),
                 _ptr(ops), _ptr(types), ctypes.cast(ptrs, ctypes.c_void_p).value,
                 _ptr(sizes), _ptr(reqlist), _ptr(mux_off), _ptr(mux_stream))
    nops = len(ops)
    match = np.full(max(1, nops), -1, np.int64)
    post = np.full(max(1, nops), -1, np.int32)
    done = np.full(max(1, nops), -1, np.int32)
    status = np.zeros(max(1, prog.nstatus), STATUS_DTYPE)
    stuck = np.full(max(1, prog.nstreams), -1, np.int32)
    R = _Result(_ptr(match), _ptr(post), _ptr(done), _ptr(status), _ptr(stuck), 0, 0, 0, 0)
    lib.oracle_run(ctypes.byref(P), ctypes.byref(R))
    return OracleOutcome(buffers=bufs, match=match[:nops], post_round=post[:nops],
                         done_round=done[:nops], status=status[:prog.nstatus],
                         stuck_op=stuck[:prog.nstreams], rounds=int(R.rounds),
                         deadlock=bool(R.deadlock), error=int(R.error))


def sum_f32_ref(xs: List[np.ndarray]):
    """Rank-order double sum and magnitude sum of R float32 vectors."""
    lib = _load()
    xs = [np.ascontiguousarray(x, np.float32) for x in xs]
    n = xs[0].size
    arr = (ctypes.c_void_p * len(xs))(*[x.ctypes.data for x in xs])
    s = np.zeros(n, np.float64)
    a = np.zeros(n, np.float64)
    lib.oracle_sum_f32_ref(len(xs), n, ctypes.cast(arr, ctypes.c_void_p), _ptr(s), _ptr(a))
    return s, a
