"""Traffic programs: a closed description of what every virtual rank enqueues.

A program lists, per MPIX stream (a serial execution context bound to one
virtual rank, §3.1), the ordered operations that stream enqueues: sends,
receives, waits, allreduces and the user compute kernels interleaved with them
(the SAXPY of Listing 4, §6).  Buffers are byte arrays referenced by
(buffer id, byte offset).  Both the CPU oracle and the GPU harness consume the
same program; this module only describes inputs and holds none of the
matching, copying or reduction logic.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

# --- operation kinds (the enqueue calls of §3.4 plus the user compute op) ---
(SEND, RECV, ISEND, IRECV, WAIT, WAITALL, ALLREDUCE, AXPY, BCAST, REDUCE, ALLGATHER,
 IALLREDUCE, IBCAST, IREDUCE, IALLGATHER) = range(15)
KIND_NAMES = ["send", "recv", "isend", "irecv", "wait", "waitall", "allreduce", "axpy",
              "bcast", "reduce", "allgather", "iallreduce", "ibcast", "ireduce", "iallgather"]
NONBLOCKING_COLLECTIVES = (IALLREDUCE, IBCAST, IREDUCE, IALLGATHER)
COLLECTIVES = (ALLREDUCE, BCAST, REDUCE, ALLGATHER) + NONBLOCKING_COLLECTIVES

ANY_SOURCE = -2
ANY_TAG = -1
ANY_INDEX = -1         # multiplex stream communicators: any of the source rank's streams
IN_PLACE = -3          # allreduce send buffer id meaning "use the receive buffer"

# --- predefined datatypes (ids 0..4); derived vector types are appended ---
T_BYTE, T_INT32, T_INT64, T_FLOAT, T_DOUBLE = range(5)
BASIC_SIZES = {T_BYTE: 1, T_INT32: 4, T_INT64: 8, T_FLOAT: 4, T_DOUBLE: 8}
BASIC_NP = {T_BYTE: np.uint8, T_INT32: np.int32, T_INT64: np.int64,
            T_FLOAT: np.float32, T_DOUBLE: np.float64}

# allreduce reduction modes
MODE_FIXED, MODE_TREE = 0, 1

# status error codes (documented interface values; see include/mpx.h)
ERR_SUCCESS = 0
ERR_TRUNCATE = 15
ERR_TIMEOUT = 16

# One record per operation.  Field order and offsets are an interface format
# shared with the oracle's C struct (88 bytes, little endian).  sidx / didx:
# on a multiplex stream communicator (§3.5) the sender's and the receiver's
# local stream index (a receive's sidx may be ANY_INDEX); 0 on other comms.
# persist: k + 1 when a nonblocking collective is a start of persistent
# request k (MPI-4 persistent collectives, e.g. MPI_Allreduce_init), else 0;
# the oracle ignores it (a start behaves as the nonblocking call it starts).
OP_DTYPE = np.dtype({
    "names": ["stream", "kind", "comm", "peer", "tag", "type", "count",
              "buf", "buf2", "off", "off2", "req_lo", "req_n", "status",
              "mode", "alpha", "sidx", "didx", "persist"],
    "formats": ["<i4", "<i4", "<i4", "<i4", "<i4", "<i4", "<i8",
                "<i4", "<i4", "<i8", "<i8", "<i4", "<i4", "<i4",
                "<i4", "<f4", "<i4", "<i4", "<i4"],
    "offsets": [0, 4, 8, 12, 16, 20, 24, 32, 36, 40, 48, 56, 60, 64, 68, 72, 76, 80, 84],
    "itemsize": 88,
})

# kind 0 = predefined, 1 = vector(vcount, blocklen, stride) of a predefined type
TYPE_DTYPE = np.dtype({
    "names": ["kind", "base", "elem", "vcount", "blocklen", "stride"],
    "formats": ["<i4"] * 6,
    "offsets": [0, 4, 8, 12, 16, 20],
    "itemsize": 24,
})

# source_index: the sender's local stream index on a multiplex comm, else 0
STATUS_DTYPE = np.dtype({
    "names": ["source", "tag", "error", "source_index", "bytes"],
    "formats": ["<i4", "<i4", "<i4", "<i4", "<i8"],
    "offsets": [0, 4, 8, 12, 16],
    "itemsize": 24,
})


def basic_types() -> np.ndarray:
    t = np.zeros(5, TYPE_DTYPE)
    for i in range(5):
        t[i] = (0, i, BASIC_SIZES[i], 1, 1, 1)
    return t


def type_size(types: np.ndarray, t: int) -> int:
    """Bytes of data in one instance of type t (gaps excluded)."""
    r = types[t]
    return int(r["elem"]) * int(r["vcount"]) * int(r["blocklen"])


def type_extent(types: np.ndarray, t: int) -> int:
    """MPI extent of one instance (lower bound 0): ((vcount-1)*stride+blocklen)*elem."""
    r = types[t]
    if r["kind"] == 0:
        return int(r["elem"])
    return ((int(r["vcount"]) - 1) * int(r["stride"]) + int(r["blocklen"])) * int(r["elem"])


def span_bytes(types: np.ndarray, t: int, count: int) -> int:
    """Bytes of memory touched by `count` instances starting at offset 0."""
    if count <= 0:
        return 0
    r = types[t]
    if r["kind"] == 0:
        return count * int(r["elem"])
    return (count - 1) * type_extent(types, t) + type_extent(types, t)


@dataclass
class Program:
    nranks: int
    stream_rank: np.ndarray            # int32 [nstreams]
    comm_stream: np.ndarray            # int32 [ncomms, nranks]
    ops: np.ndarray                    # OP_DTYPE [nops], grouped by stream
    stream_op_lo: np.ndarray           # int64 [nstreams + 1]
    types: np.ndarray                  # TYPE_DTYPE
    buf_init: List[np.ndarray]         # uint8 initial contents per buffer
    reqlist: np.ndarray                # int64 op indices used by wait/waitall
    nstatus: int
    issue_order: np.ndarray            # int64 op indices in host enqueue order
    name: str = ""
    meta: dict = field(default_factory=dict)
    # per comm: None, or (multiplex stream comm, §3.5) per rank the list of its
    # local streams in index order; comm_stream then holds each rank's index 0
    comm_mux: List[Optional[List[List[int]]]] = field(default_factory=list)

    def mux(self, c: int) -> Optional[List[List[int]]]:
        return self.comm_mux[c] if c < len(self.comm_mux) else None

    def member(self, c: int, g: int):
        """(rank, local index) of stream g in comm c, or None."""
        m = self.mux(c)
        if m is None:
            hits = np.nonzero(self.comm_stream[c] == g)[0]
            return (int(hits[0]), 0) if len(hits) else None
        for r, lst in enumerate(m):
            if g in lst:
                return (r, lst.index(g))
        return None

    @property
    def nstreams(self) -> int:
        return len(self.stream_rank)

    @property
    def ncomms(self) -> int:
        return self.comm_stream.shape[0]

    def fresh_buffers(self) -> List[np.ndarray]:
        return [b.copy() for b in self.buf_init]


class ProgramBuilder:
    """Accumulates per-stream operation lists in program order."""

    def __init__(self, nranks: int, name: str = ""):
        self.nranks = nranks
        self.name = name
        self.stream_rank: List[int] = []
        self.comms: List[List[int]] = []
        self.comm_mux: List[Optional[List[List[int]]]] = []
        self.per_stream: List[List[dict]] = []
        self.types = list(basic_types())
        self.bufs: List[np.ndarray] = []
        self.nstatus = 0
        self.issue: List[tuple] = []
        self.meta: dict = {}
        self.persistents: List[dict] = []

    # --- objects ---
    def stream(self, rank: int) -> int:
        assert 0 <= rank < self.nranks
        self.stream_rank.append(rank)
        self.per_stream.append([])
        return len(self.stream_rank) - 1

    def comm(self, streams: Sequence[int]) -> int:
        assert len(streams) == self.nranks
        for r, g in enumerate(streams):
            assert self.stream_rank[g] == r, "comm member r must be a stream of rank r"
        self.comms.append(list(streams))
        self.comm_mux.append(None)
        return len(self.comms) - 1

    def comm_multiple(self, local_streams: Sequence[Sequence[int]]) -> int:
        """MPIX_Stream_comm_create_multiple (§3.5): rank r attaches the streams
        local_streams[r] (at least one), addressed by their index in that list."""
        assert len(local_streams) == self.nranks
        lists = []
        for r, lst in enumerate(local_streams):
            assert len(lst) >= 1 and len(set(lst)) == len(lst)
            for g in lst:
                assert self.stream_rank[g] == r, "rank r attaches streams of rank r"
            lists.append(list(lst))
        self.comms.append([lst[0] for lst in lists])
        self.comm_mux.append(lists)
        return len(self.comms) - 1

    def _index(self, comm: int, g: int) -> int:
        lists = self.comm_mux[comm]
        assert lists is not None, "a multiplex stream communicator"
        return lists[self.stream_rank[g]].index(g)

    def vector(self, vcount: int, blocklen: int, stride: int, base: int) -> int:
        assert base in BASIC_SIZES and vcount >= 1 and blocklen >= 1 and stride >= blocklen
        rec = np.zeros(1, TYPE_DTYPE)[0]
        rec["kind"], rec["base"], rec["elem"] = 1, base, BASIC_SIZES[base]
        rec["vcount"], rec["blocklen"], rec["stride"] = vcount, blocklen, stride
        self.types.append(rec)
        return len(self.types) - 1

    def buffer(self, init) -> int:
        """init: an int byte count (zero-filled) or a uint8/any numpy array."""
        if isinstance(init, (int, np.integer)):
            arr = np.zeros(int(init), np.uint8)
        else:
            arr = np.ascontiguousarray(init).view(np.uint8).reshape(-1).copy()
        self.bufs.append(arr)
        return len(self.bufs) - 1

    def status_slots(self, n: int) -> int:
        base = self.nstatus
        self.nstatus += n
        return base

    # --- operations ---
    def _op(self, g: int, **kw) -> tuple:
        rec = dict(stream=g, kind=0, comm=-1, peer=0, tag=0, type=0, count=0,
                   buf=-1, buf2=-1, off=0, off2=0, req_lo=0, req_n=0,
                   status=-1, mode=0, alpha=0.0, sidx=0, didx=0, reqs=None)
        rec.update(kw)
        self.per_stream[g].append(rec)
        h = (g, len(self.per_stream[g]) - 1)
        self.issue.append(h)
        return h

    def send(self, g, comm, buf, off, count, type_, dest, tag):
        return self._op(g, kind=SEND, comm=comm, buf=buf, off=off, count=count,
                        type=type_, peer=dest, tag=tag)

    def isend(self, g, comm, buf, off, count, type_, dest, tag):
        return self._op(g, kind=ISEND, comm=comm, buf=buf, off=off, count=count,
                        type=type_, peer=dest, tag=tag)

    def recv(self, g, comm, buf, off, count, type_, source, tag, status=-1):
        return self._op(g, kind=RECV, comm=comm, buf=buf, off=off, count=count,
                        type=type_, peer=source, tag=tag, status=status)

    def irecv(self, g, comm, buf, off, count, type_, source, tag):
        return self._op(g, kind=IRECV, comm=comm, buf=buf, off=off, count=count,
                        type=type_, peer=source, tag=tag)

    # MPIX_Stream_send / recv / isend / irecv (§3.5): stream g is the caller's
    # local stream (src_idx for sends, dst_idx for receives)
    def stream_send(self, g, comm, buf, off, count, type_, dest, dst_idx, tag, blocking=False):
        return self._op(g, kind=SEND if blocking else ISEND, comm=comm, buf=buf, off=off,
                        count=count, type=type_, peer=dest, tag=tag,
                        sidx=self._index(comm, g), didx=dst_idx)

    def stream_recv(self, g, comm, buf, off, count, type_, source, src_idx, tag, blocking=False,
                    status=-1):
        return self._op(g, kind=RECV if blocking else IRECV, comm=comm, buf=buf, off=off,
                        count=count, type=type_, peer=source, tag=tag, status=status,
                        sidx=src_idx, didx=self._index(comm, g))

    def wait(self, g, req, status=-1):
        assert req[0] == g
        return self._op(g, kind=WAIT, reqs=[req], status=status)

    def waitall(self, g, reqs, status_base=-1):
        for r in reqs:
            assert r[0] == g, "waitall requests must share one stream (§3.4)"
        return self._op(g, kind=WAITALL, reqs=list(reqs), status=status_base)

    def allreduce(self, g, comm, sendbuf, sendoff, recvbuf, recvoff, count, type_,
                  mode=MODE_FIXED):
        return self._op(g, kind=ALLREDUCE, comm=comm, buf=sendbuf, off=sendoff,
                        buf2=recvbuf, off2=recvoff, count=count, type=type_, mode=mode)

    def bcast(self, g, comm, buf, off, count, type_, root):
        """MPI_Bcast: the root's count elements replace every other rank's."""
        return self._op(g, kind=BCAST, comm=comm, buf=buf, off=off, count=count, type=type_,
                        peer=root)

    def reduce(self, g, comm, sendbuf, sendoff, recvbuf, recvoff, count, type_, root,
               mode=MODE_FIXED):
        """MPI_Reduce (SUM) to `root`; recvbuf matters at the root only (-1 elsewhere);
        sendbuf IN_PLACE at the root reduces its receive buffer."""
        return self._op(g, kind=REDUCE, comm=comm, buf=sendbuf, off=sendoff, buf2=recvbuf,
                        off2=recvoff, count=count, type=type_, peer=root, mode=mode)

    def allgather(self, g, comm, sendbuf, sendoff, recvbuf, recvoff, count, type_):
        """MPI_Allgather: count elements per rank into R blocks of every receive
        buffer; sendbuf IN_PLACE: the rank's block is already in place."""
        return self._op(g, kind=ALLGATHER, comm=comm, buf=sendbuf, off=sendoff, buf2=recvbuf,
                        off2=recvoff, count=count, type=type_)

    # nonblocking forms (MPI_Iallreduce, ...): the handle goes to wait / waitall
    def iallreduce(self, g, comm, sendbuf, sendoff, recvbuf, recvoff, count, type_,
                   mode=MODE_FIXED):
        return self._op(g, kind=IALLREDUCE, comm=comm, buf=sendbuf, off=sendoff,
                        buf2=recvbuf, off2=recvoff, count=count, type=type_, mode=mode)

    def ibcast(self, g, comm, buf, off, count, type_, root):
        return self._op(g, kind=IBCAST, comm=comm, buf=buf, off=off, count=count, type=type_,
                        peer=root)

    def ireduce(self, g, comm, sendbuf, sendoff, recvbuf, recvoff, count, type_, root,
                mode=MODE_FIXED):
        return self._op(g, kind=IREDUCE, comm=comm, buf=sendbuf, off=sendoff, buf2=recvbuf,
                        off2=recvoff, count=count, type=type_, peer=root, mode=mode)

    def iallgather(self, g, comm, sendbuf, sendoff, recvbuf, recvoff, count, type_):
        return self._op(g, kind=IALLGATHER, comm=comm, buf=sendbuf, off=sendoff, buf2=recvbuf,
                        off2=recvoff, count=count, type=type_)

    # --- persistent collectives (MPI-4: MPI_Allreduce_init / MPI_Start) ---
    def persistent(self, g, kind, comm, **args) -> int:
        """A persistent request on stream g for the nonblocking collective
        `kind` (IALLREDUCE, IBCAST, IREDUCE or IALLGATHER) with fixed
        arguments (the builder method's keywords).  Records no operation: the
        request only names what each start() enqueues.  Returns its id."""
        assert kind in NONBLOCKING_COLLECTIVES
        self.persistents.append(dict(g=g, kind=kind, comm=comm, args=dict(args)))
        return len(self.persistents) - 1

    def start(self, g, pid):
        """Start persistent request pid: its nonblocking collective, enqueued
        here on g; completed by a wait like any request."""
        p = self.persistents[pid]
        assert p["g"] == g, "a persistent request is started on the stream that created it"
        return self._op(g, kind=p["kind"], comm=p["comm"], persist=pid + 1, **p["args"])

    def axpy(self, g, alpha, xbuf, xoff, ybuf, yoff, n):
        """y[i] = alpha*x[i] + y[i] in fp32 with one rounding (fused multiply-add)."""
        return self._op(g, kind=AXPY, alpha=alpha, buf=xbuf, off=xoff, buf2=ybuf,
                        off2=yoff, count=n, type=T_FLOAT)

    # --- finish ---
    def build(self) -> Program:
        ns = len(self.stream_rank)
        lo = np.zeros(ns + 1, np.int64)
        for g in range(ns):
            lo[g + 1] = lo[g] + len(self.per_stream[g])
        nops = int(lo[-1])
        ops = np.zeros(nops, OP_DTYPE)
        reqlist: List[int] = []
        for g in range(ns):
            for i, rec in enumerate(self.per_stream[g]):
                j = int(lo[g]) + i
                reqs = rec.pop("reqs")
                if reqs is not None:
                    rec["req_lo"] = len(reqlist)
                    rec["req_n"] = len(reqs)
                    for (rg, ri) in reqs:
                        reqlist.append(int(lo[rg]) + ri)
                for k, v in rec.items():
                    ops[j][k] = v
                rec["reqs"] = reqs
        issue = np.array([int(lo[g]) + i for (g, i) in self.issue], np.int64)
        comm_stream = (np.array(self.comms, np.int32).reshape(len(self.comms), self.nranks)
                       if self.comms else np.zeros((0, self.nranks), np.int32))
        return Program(nranks=self.nranks,
                       stream_rank=np.array(self.stream_rank, np.int32),
                       comm_stream=comm_stream, ops=ops, stream_op_lo=lo,
                       types=np.array(self.types, TYPE_DTYPE),
                       buf_init=self.bufs, reqlist=np.array(reqlist, np.int64),
                       nstatus=self.nstatus, issue_order=issue, name=self.name,
                       meta=dict(self.meta, persistents=[dict(p) for p in self.persistents]),
                       comm_mux=[None if m is None else [list(l) for l in m]
                                 for m in self.comm_mux])
