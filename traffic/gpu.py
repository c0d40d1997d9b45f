"""Run a traffic program on the GPU through libmpx's C ABI.

Device memory and CUDA streams come from PyTorch; every operation goes
through the library (`paper_2208_13707_gb300.mpx`), and the user compute op
(axpy) through the library's exported Listing 4 kernel.  Nothing here
computes a result: it allocates, enqueues in the program's issue order,
waits with a host-side deadline, and reads buffers and statuses back.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from .program import (ALLGATHER, ALLREDUCE, AXPY, BCAST, IALLGATHER, IALLREDUCE, IBCAST, IN_PLACE,
                      IRECV, IREDUCE, ISEND, RECV, REDUCE, SEND, STATUS_DTYPE, WAIT, WAITALL,
                      Program)


@dataclass
class GpuOutcome:
    buffers: List[np.ndarray]
    status: np.ndarray
    stream_errors: List[int]
    world_error: int
    counters: List[int]
    finished: bool
    seconds: float
    extra: dict = field(default_factory=dict)


def _pow2_at_least(n: int, lo: int) -> int:
    v = lo
    while v < n:
        v *= 2
    return v


def make_config(prog: Program, mode: int, **over):
    from paper_2208_13707_gb300 import mpx
    cfg = mpx.mpx_world_config_init()
    cfg.engine_mode = mode
    cfg.max_streams = max(cfg.max_streams, prog.nstreams)
    per_stream = int(np.max(np.diff(prog.stream_op_lo))) if prog.nstreams else 1
    cfg.ring_slots = _pow2_at_least(per_stream + 1, 256)
    # a multiplex comm of M members takes ceil(M / nranks) comm slots
    slots = 0
    for c in range(prog.ncomms):
        m = prog.mux(c)
        members = prog.nranks if m is None else sum(len(l) for l in m)
        slots += -(-members // prog.nranks)
    cfg.max_comms = max(1, slots)
    cfg.queue_slots = _pow2_at_least(per_stream + 1, 256)
    cfg.watchdog_ns = int(5e9)
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


def run(prog: Program, mode: str = "persistent", timeout_s: float = 60.0, exclusive: bool = False,
        cfg_over: Optional[dict] = None, buffers: Optional[list] = None, keep_world: bool = False,
        drain_passes: int = 10000) -> GpuOutcome:
    import torch
    from paper_2208_13707_gb300 import mpx
    dev = torch.device("cuda")
    m = {"persistent": mpx.ENGINE_PERSISTENT, "drain": mpx.ENGINE_DRAIN, "plain": mpx.ENGINE_PLAIN}[mode]
    cfg = make_config(prog, m, **(cfg_over or {}))
    init = buffers if buffers is not None else prog.buf_init
    dbufs = [torch.from_numpy(np.ascontiguousarray(b)).to(dev) if b.size else
             torch.empty(16, dtype=torch.uint8, device=dev) for b in init]
    st = torch.zeros(max(1, prog.nstatus) * STATUS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    torch.cuda.current_stream(dev).synchronize()
    ptr = [b.data_ptr() for b in dbufs]
    st_ptr = st.data_ptr()

    def sptr(slot):
        return 0 if slot < 0 else st_ptr + STATUS_DTYPE.itemsize * int(slot)

    world = mpx.mpx_world_create(prog.nranks, cfg)
    # distinct non-blocking streams (torch.cuda.Stream() hands out a fixed pool)
    raw_streams = [mpx.mpx_cuda_stream_create() for _ in range(prog.nstreams + 1)]
    cstreams = [torch.cuda.ExternalStream(h, device=dev) for h in raw_streams[:-1]]
    flags = mpx.STREAM_EXCLUSIVE if exclusive else mpx.STREAM_DEFAULT
    ms = []
    for g in range(prog.nstreams):
        ms.append(mpx.mpx_stream_create(world, int(prog.stream_rank[g]), cstreams[g].cuda_stream, flags))
        assert mpx.mpx_stream_get_id(ms[g]) == g
    comms = [mpx.mpx_stream_comm_create(world, [ms[int(g)] for g in prog.comm_stream[c]])
             if prog.mux(c) is None else
             mpx.mpx_stream_comm_create_multiple(world, [[ms[int(g)] for g in l] for l in prog.mux(c)])
             for c in range(prog.ncomms)]
    tmap = {}
    for t in range(len(prog.types)):
        r = prog.types[t]
        tmap[t] = t if t < 5 else mpx.mpx_type_vector(int(r["vcount"]), int(r["blocklen"]),
                                                      int(r["stride"]), int(r["base"]))
    rank_in = {}
    for c in range(prog.ncomms):
        for r, g in enumerate(prog.comm_stream[c]):
            rank_in[(c, int(g))] = r
        for r, l in enumerate(prog.mux(c) or []):
            for g in l:
                rank_in[(c, int(g))] = r
    engine_stream = torch.cuda.ExternalStream(raw_streams[-1], device=dev)
    req: Dict[int, int] = {}
    persist: Dict[int, int] = {}   # persistent request id -> handle (created at its first start)
    ops = prog.ops

    def retry(fn):
        for _ in range(100000):
            try:
                return fn()
            except mpx.MpxError as e:
                if e.code != mpx.ERR_AGAIN:
                    raise
                if m == mpx.ENGINE_DRAIN:
                    mpx.mpx_world_progress(world, engine_stream.cuda_stream)
                    t_dl = time.perf_counter() + timeout_s
                    while not engine_stream.query() and time.perf_counter() < t_dl:
                        time.sleep(5e-5)
                else:
                    time.sleep(1e-4)
        raise RuntimeError("submission ring stayed full")

    def issue(j):
        o = ops[int(j)]
        k, g = int(o["kind"]), int(o["stream"])
        c = int(o["comm"])
        comm = comms[c][rank_in[(c, g)]] if c >= 0 else None
        b = int(o["buf"])
        p = ptr[b] + int(o["off"]) if b >= 0 else 0
        cnt, ty, peer, tag = int(o["count"]), tmap.get(int(o["type"]), 0), int(o["peer"]), int(o["tag"])
        si, di = int(o["sidx"]), int(o["didx"])
        if c >= 0 and prog.mux(c) is not None:  # MPIX_Stream_* on a multiplex comm (§3.5)
            if k == SEND:
                retry(lambda: mpx.mpx_stream_send_enqueue(p, cnt, ty, peer, tag, comm, si, di))
            elif k == RECV:
                retry(lambda: mpx.mpx_stream_recv_enqueue(p, cnt, ty, peer, tag, comm, si, di,
                                                          sptr(int(o["status"]))))
            elif k == ISEND:
                req[int(j)] = retry(lambda: mpx.mpx_stream_isend_enqueue(p, cnt, ty, peer, tag, comm,
                                                                         si, di))
            elif k == IRECV:
                req[int(j)] = retry(lambda: mpx.mpx_stream_irecv_enqueue(p, cnt, ty, peer, tag, comm,
                                                                         si, di))
            else:
                raise ValueError(f"kind {k} on a multiplex comm")
        elif k == SEND:
            retry(lambda: mpx.mpx_send_enqueue(p, cnt, ty, peer, tag, comm))
        elif k == RECV:
            retry(lambda: mpx.mpx_recv_enqueue(p, cnt, ty, peer, tag, comm, sptr(int(o["status"]))))
        elif k == ISEND:
            req[int(j)] = retry(lambda: mpx.mpx_isend_enqueue(p, cnt, ty, peer, tag, comm))
        elif k == IRECV:
            req[int(j)] = retry(lambda: mpx.mpx_irecv_enqueue(p, cnt, ty, peer, tag, comm))
        elif k in (WAIT, WAITALL):
            lo, n = int(o["req_lo"]), int(o["req_n"])
            hs = [req[int(q)] for q in prog.reqlist[lo: lo + n]]
            if k == WAIT:
                retry(lambda: mpx.mpx_wait_enqueue(hs[0], sptr(int(o["status"]))))
            else:
                retry(lambda: mpx.mpx_waitall_enqueue(hs, sptr(int(o["status"]))))
        elif k == ALLREDUCE:
            rb = ptr[int(o["buf2"])] + int(o["off2"]) if int(o["buf2"]) >= 0 else 0
            sb = mpx.IN_PLACE if b == IN_PLACE else p
            retry(lambda: mpx.mpx_allreduce_enqueue(sb, rb, cnt, ty, mpx.SUM, comm))
        elif k == BCAST:
            retry(lambda: mpx.mpx_bcast_enqueue(p, cnt, ty, peer, comm))
        elif k == REDUCE:
            b2 = int(o["buf2"])
            rb = ptr[b2] + int(o["off2"]) if b2 >= 0 else 0
            sb = mpx.IN_PLACE if b == IN_PLACE else p
            retry(lambda: mpx.mpx_reduce_enqueue(sb, rb, cnt, ty, mpx.SUM, peer, comm))
        elif k == ALLGATHER:
            rb = ptr[int(o["buf2"])] + int(o["off2"])
            sb = mpx.IN_PLACE if b == IN_PLACE else p
            retry(lambda: mpx.mpx_allgather_enqueue(sb, rb, cnt, ty, comm))
        elif int(o["persist"]) > 0:
            # a start of a persistent collective: its init call at the first start
            pid = int(o["persist"]) - 1
            if pid not in persist:
                b2 = int(o["buf2"])
                rb = ptr[b2] + int(o["off2"]) if b2 >= 0 else 0
                sb = mpx.IN_PLACE if b == IN_PLACE else p
                persist[pid] = {IALLREDUCE: lambda: mpx.mpx_allreduce_init(sb, rb, cnt, ty, mpx.SUM, comm),
                                IBCAST: lambda: mpx.mpx_bcast_init(p, cnt, ty, peer, comm),
                                IREDUCE: lambda: mpx.mpx_reduce_init(sb, rb, cnt, ty, mpx.SUM, peer, comm),
                                IALLGATHER: lambda: mpx.mpx_allgather_init(sb, rb, cnt, ty, comm)}[k]()
            retry(lambda: mpx.mpx_start_enqueue(persist[pid]))
            req[int(j)] = persist[pid]
        elif k == IALLREDUCE:
            rb = ptr[int(o["buf2"])] + int(o["off2"]) if int(o["buf2"]) >= 0 else 0
            sb = mpx.IN_PLACE if b == IN_PLACE else p
            req[int(j)] = retry(lambda: mpx.mpx_iallreduce_enqueue(sb, rb, cnt, ty, mpx.SUM, comm))
        elif k == IBCAST:
            req[int(j)] = retry(lambda: mpx.mpx_ibcast_enqueue(p, cnt, ty, peer, comm))
        elif k == IREDUCE:
            b2 = int(o["buf2"])
            rb = ptr[b2] + int(o["off2"]) if b2 >= 0 else 0
            sb = mpx.IN_PLACE if b == IN_PLACE else p
            req[int(j)] = retry(lambda: mpx.mpx_ireduce_enqueue(sb, rb, cnt, ty, mpx.SUM, peer, comm))
        elif k == IALLGATHER:
            rb = ptr[int(o["buf2"])] + int(o["off2"])
            sb = mpx.IN_PLACE if b == IN_PLACE else p
            req[int(j)] = retry(lambda: mpx.mpx_iallgather_enqueue(sb, rb, cnt, ty, comm))
        elif k == AXPY:
            yb = ptr[int(o["buf2"])] + int(o["off2"])
            mpx.mpx_saxpy_enqueue(cnt, float(o["alpha"]), p, yb, cstreams[g].cuda_stream)
        else:
            raise ValueError(k)

    t0 = time.perf_counter()
    if m != mpx.ENGINE_PLAIN:
        for j in prog.issue_order:
            issue(j)
    else:
        # the plain path completes calls on the host; a blocking call that
        # cannot complete yet answers MPX_ERR_AGAIN: move on to other streams
        retry = lambda fn: fn()
        lo = prog.stream_op_lo
        cur = [int(lo[g]) for g in range(prog.nstreams)]
        idle_since = time.perf_counter()
        while any(cur[g] < int(lo[g + 1]) for g in range(prog.nstreams)):
            moved = False
            for g in range(prog.nstreams):
                while cur[g] < int(lo[g + 1]):
                    try:
                        issue(cur[g])
                    except mpx.MpxError as e:
                        if e.code != mpx.ERR_AGAIN:
                            raise
                        break
                    cur[g] += 1
                    moved = True
            if moved:
                idle_since = time.perf_counter()
            elif time.perf_counter() - idle_since > timeout_s:
                raise RuntimeError("plain path made no progress (deadlocked program?)")
    t_issue = time.perf_counter() - t0

    deadline = time.perf_counter() + timeout_s
    finished = False
    passes = 0
    if m == mpx.ENGINE_DRAIN:
        while time.perf_counter() < deadline and passes < drain_passes:
            mpx.mpx_world_progress(world, engine_stream.cuda_stream)
            while not engine_stream.query() and time.perf_counter() < deadline:
                time.sleep(5e-5)
            passes += 1
            if all(mpx.mpx_stream_pending(s) == 0 for s in ms):
                break
            if passes % 200 == 0 and all(s.query() for s in cstreams):
                # the streams are idle yet operations stay pending: report
                import sys
                print(f"[gpu.run] drain: streams idle, pending "
                      f"{[mpx.mpx_stream_pending(s) for s in ms]}", file=sys.stderr, flush=True)
                mpx.mpx_world_debug_dump(world)
                break
    while time.perf_counter() < deadline:
        if all(s.query() for s in cstreams):
            finished = True
            break
        time.sleep(1e-4)
    seconds = time.perf_counter() - t0
    if not finished or (m == mpx.ENGINE_DRAIN and passes >= drain_passes):
        import sys
        print(f"[gpu.run] deadline: finished={finished} passes={passes} counters="
              f"{mpx.mpx_world_get_counters(world)}", file=sys.stderr, flush=True)
        if m != mpx.ENGINE_PLAIN:
            mpx.mpx_world_debug_dump(world)
    if not finished:
        # release every waiter so the streams drain, then give them a moment
        mpx.mpx_world_abort(world)
        t1 = time.perf_counter()
        while time.perf_counter() - t1 < 10 and not all(s.query() for s in cstreams):
            time.sleep(1e-3)
    out_bufs = [b.cpu().numpy()[: init[i].size].copy() for i, b in enumerate(dbufs)] if finished else []
    status = np.frombuffer(st.cpu().numpy().tobytes(), STATUS_DTYPE)[: prog.nstatus].copy() if finished else None
    serr = [mpx.mpx_stream_get_error(s) for s in ms]
    werr = mpx.mpx_world_get_error(world)
    counters = mpx.mpx_world_get_counters(world)
    extra = {"issue_seconds": t_issue, "drain_passes": passes}
    if finished:
        for h in persist.values():  # every start was waited for: the requests are inactive
            mpx.mpx_request_free(h)
    if finished and not keep_world:
        for c in range(prog.ncomms):
            for h in comms[c]:
                mpx.mpx_comm_free(h)
        for t, v in tmap.items():
            if t >= 5:
                mpx.mpx_type_free(v)
        for s in ms:
            for _ in range(2000):
                try:
                    mpx.mpx_stream_free(s)
                    break
                except mpx.MpxError as e:
                    if e.code != mpx.ERR_PENDING:
                        raise
                    time.sleep(5e-4)
            else:
                raise RuntimeError("stream still has pending operations")
        mpx.mpx_world_free(world)
        for h in raw_streams:
            mpx.mpx_cuda_stream_destroy(h)
    elif keep_world:
        extra.update(world=world, streams=ms, comms=comms, cstreams=cstreams, dbufs=dbufs)
    return GpuOutcome(buffers=out_bufs, status=status, stream_errors=serr, world_error=werr,
                      counters=counters, finished=finished, seconds=seconds, extra=extra)


class BatchRunner:
    """A closed program in which every stream's only blocking operation is its
    last one (a waitall over all of the stream's requests), run repeatedly
    through mpx_enqueue_batch: one call enqueues every stream's non-blocking
    operations, then every stream's waitall.  A stream may begin with axpy
    compute ops (Listing 4's kernel): they are launched on the stream before
    its communication, and a recorded step is ordered after them.  Holds the
    world, streams, buffers and the prebuilt operation array between steps."""

    def __init__(self, prog: Program, mode: str = "persistent", exclusive: bool = True,
                 cfg_over: Optional[dict] = None, timeout_s: float = 60.0,
                 epoch_barrier: bool = False):
        """epoch_barrier: end every stream's step with a one-element in-place
        allreduce on the stream's comm, so that steps enqueued back to back
        stay separate epochs (a stream's next step posts nothing before every
        member of its comm has finished this one).  Not for the plain path,
        whose blocking allreduce cannot wait inside one batch call."""
        import torch
        from paper_2208_13707_gb300 import mpx
        self.mpx, self.torch, self.prog, self.timeout_s = mpx, torch, prog, timeout_s
        dev = torch.device("cuda")
        # "graph": the step is recorded once (mpx_step_create, drain-mode world)
        # and every step() replays its CUDA graph on the engine stream
        self.graph = mode == "graph"
        self.mode = {"persistent": mpx.ENGINE_PERSISTENT, "drain": mpx.ENGINE_DRAIN,
                     "plain": mpx.ENGINE_PLAIN, "graph": mpx.ENGINE_DRAIN}[mode]
        over = {"task_slots": 1 << 16}
        over.update(cfg_over or {})
        cfg = make_config(prog, self.mode, **over)
        self.dbufs = [torch.from_numpy(np.ascontiguousarray(b)).to(dev) if b.size else
                      torch.empty(16, dtype=torch.uint8, device=dev) for b in prog.buf_init]
        self.st = torch.zeros(max(1, prog.nstatus) * STATUS_DTYPE.itemsize, dtype=torch.uint8,
                              device=dev)
        torch.cuda.current_stream(dev).synchronize()
        self.world = mpx.mpx_world_create(prog.nranks, cfg)
        self.raw = [mpx.mpx_cuda_stream_create() for _ in range(prog.nstreams + 1)]
        self.cstreams = [torch.cuda.ExternalStream(h, device=dev) for h in self.raw[:-1]]
        self.engine_stream = torch.cuda.ExternalStream(self.raw[-1], device=dev)
        flags = mpx.STREAM_EXCLUSIVE if exclusive else mpx.STREAM_DEFAULT
        self.ms = [mpx.mpx_stream_create(self.world, int(prog.stream_rank[g]),
                                         self.cstreams[g].cuda_stream, flags)
                   for g in range(prog.nstreams)]
        self.comms = [mpx.mpx_stream_comm_create(self.world, [self.ms[int(g)] for g in prog.comm_stream[c]])
                      for c in range(prog.ncomms)]
        self.tmap = np.array([t if t < 5 else mpx.mpx_type_vector(
            int(prog.types[t]["vcount"]), int(prog.types[t]["blocklen"]),
            int(prog.types[t]["stride"]), int(prog.types[t]["base"]))
            for t in range(len(prog.types))], np.int32)
        self.epoch_barrier = epoch_barrier
        if epoch_barrier:
            assert self.mode != mpx.ENGINE_PLAIN
            self.bar = torch.zeros(prog.nstreams * 4, dtype=torch.int32, device=dev)
            torch.cuda.synchronize()
        self.ops = self._build_ops()
        # an exclusive stream has no doorbell: the engine takes its operations
        # as reached at once, which a compute op ahead of them would break
        assert not (self.axpys and exclusive and not self.graph), \
            "leading compute ops need doorbells (non-exclusive streams) or a recorded step"
        self.messages = int((np.isin(prog.ops["kind"], [SEND, ISEND])).sum())
        self.step_handle = mpx.mpx_step_create(self.world, self.ops) if self.graph else None

    def _build_ops(self):
        mpx, prog = self.mpx, self.prog
        ops = prog.ops
        nops = len(ops)
        self.reqs = np.full(nops, -1, np.int64)
        req_base = self.reqs.ctypes.data
        ptr = np.array([b.data_ptr() for b in self.dbufs], np.uint64)
        st_ptr = self.st.data_ptr()
        rank_in = {}
        for c in range(prog.ncomms):
            for r, g in enumerate(prog.comm_stream[c]):
                rank_in[(c, int(g))] = r
        comm_h = np.array([self.comms[int(o["comm"])][rank_in[(int(o["comm"]), int(o["stream"]))]]
                           if o["comm"] >= 0 else 0 for o in ops], np.uint64)
        out = np.zeros(nops, mpx.op_dtype())
        kind = ops["kind"].astype(np.int64)
        lo = prog.stream_op_lo
        nb_idx, wait_idx = [], []
        self.axpys = []  # (stream, n, alpha, x pointer, y pointer): leading compute ops
        for g in range(prog.nstreams):
            a, b = int(lo[g]), int(lo[g + 1])
            while a < b and kind[a] == AXPY:
                o = ops[a]
                self.axpys.append((g, int(o["count"]), float(o["alpha"]),
                                   int(ptr[int(o["buf"])]) + int(o["off"]),
                                   int(ptr[int(o["buf2"])]) + int(o["off2"])))
                a += 1
            if b == a:
                continue
            assert kind[b - 1] == WAITALL and np.isin(kind[a:b - 1], [ISEND, IRECV]).all(), \
                "each stream must be non-blocking operations followed by one waitall"
            q = prog.reqlist[int(ops[b - 1]["req_lo"]): int(ops[b - 1]["req_lo"]) + int(ops[b - 1]["req_n"])]
            assert np.array_equal(q, np.arange(a, b - 1)), "the waitall must cover the stream's requests in order"
            nb_idx.extend(range(a, b - 1))
            wait_idx.append(b - 1)
        order = np.array(nb_idx + wait_idx, np.int64)
        o = ops[order]
        k = kind[order]
        rec = out[: len(order)]
        rec["kind"] = np.where(k == ISEND, mpx.OP_ISEND, np.where(k == IRECV, mpx.OP_IRECV, mpx.OP_WAITALL))
        rec["datatype"] = self.tmap[o["type"]]
        rec["peer"] = o["peer"]
        rec["tag"] = o["tag"]
        bufp = np.where(o["buf"] >= 0, ptr[np.maximum(o["buf"], 0)] + o["off"].astype(np.uint64), 0)
        rec["buf"] = np.where(k == WAITALL, 0, bufp)
        rec["comm"] = comm_h[order]
        isw = k == WAITALL
        rec["count"] = np.where(isw, o["req_n"], o["count"])
        first_req = np.where(isw, order - o["req_n"], order)
        rec["requests"] = req_base + 8 * first_req.astype(np.uint64)
        rec["status"] = np.where(isw & (o["status"] >= 0),
                                 st_ptr + STATUS_DTYPE.itemsize * np.maximum(o["status"], 0).astype(np.uint64), 0)
        out = out[: len(order)].copy()
        if self.epoch_barrier:
            bar = np.zeros(prog.nstreams, mpx.op_dtype())
            bar["kind"] = mpx.OP_ALLREDUCE
            bar["datatype"] = mpx.INT32
            bar["count"] = 1
            bar["op"] = mpx.SUM
            bar["buf"] = mpx.IN_PLACE
            bar["recvbuf"] = self.bar.data_ptr() + 16 * np.arange(prog.nstreams, dtype=np.uint64)
            stream_comm = {}
            for c in range(prog.ncomms):
                for r, g in enumerate(prog.comm_stream[c]):
                    stream_comm.setdefault(int(g), self.comms[c][r])
            bar["comm"] = [stream_comm[g] for g in range(prog.nstreams)]
            out = np.concatenate([out, bar])
        return out

    def _launch_axpys(self):
        """The streams' leading compute ops; in graph mode the engine stream
        (which replays the recorded step) waits for them."""
        if not self.axpys:
            return
        for g, n, alpha, xp, yp in self.axpys:
            self.mpx.mpx_saxpy_enqueue(n, alpha, xp, yp, self.cstreams[g].cuda_stream)
        if self.graph:
            for g in sorted({a[0] for a in self.axpys}):
                self.engine_stream.wait_stream(self.cstreams[g])

    def enqueue(self):
        """Enqueue one step (returns once every operation is enqueued)."""
        mpx = self.mpx
        self._launch_axpys()
        if self.graph:
            mpx.mpx_step_launch(self.step_handle, self.engine_stream.cuda_stream)
            return
        done = 0
        n = len(self.ops)
        t_dl = time.perf_counter() + self.timeout_s
        while done < n:
            try:
                done += mpx.mpx_enqueue_batch(self.ops[done:])
            except mpx.MpxError as e:
                if e.code != mpx.ERR_AGAIN:
                    raise
                done += e.done
                if self.mode == mpx.ENGINE_PLAIN and e.done == 0:
                    # nothing else runs while this thread retries: it cannot clear
                    raise RuntimeError("plain path cannot proceed (staging arena full?)")
                if time.perf_counter() > t_dl:
                    raise RuntimeError("batch enqueue made no progress")
                if self.mode == mpx.ENGINE_DRAIN:
                    self.progress_once()
                else:
                    time.sleep(1e-5)

    def progress_once(self):
        self.mpx.mpx_world_progress(self.world, self.engine_stream.cuda_stream)

    def finish(self) -> bool:
        """Drive (drain mode) and wait until every stream is idle."""
        mpx = self.mpx
        t_dl = time.perf_counter() + self.timeout_s
        if self.graph:
            while time.perf_counter() < t_dl:
                if self.engine_stream.query():
                    return True
                time.sleep(2e-5)
            return False
        if self.mode == mpx.ENGINE_DRAIN:
            while time.perf_counter() < t_dl:
                self.progress_once()
                while not self.engine_stream.query() and time.perf_counter() < t_dl:
                    time.sleep(2e-5)
                if all(mpx.mpx_stream_pending(s) == 0 for s in self.ms):
                    break
        while time.perf_counter() < t_dl:
            if all(s.query() for s in self.cstreams):
                return True
            time.sleep(2e-5)
        import sys
        print(f"[BatchRunner] deadline: counters={mpx.mpx_world_get_counters(self.world)}",
              file=sys.stderr, flush=True)
        if self.mode != mpx.ENGINE_PLAIN:
            mpx.mpx_world_debug_dump(self.world)
        return False

    def step(self) -> bool:
        self.enqueue()
        return self.finish()

    def results(self):
        bufs = [b.cpu().numpy()[: self.prog.buf_init[i].size].copy() for i, b in enumerate(self.dbufs)]
        status = np.frombuffer(self.st.cpu().numpy().tobytes(), STATUS_DTYPE)[: self.prog.nstatus].copy()
        return bufs, status

    def reset_buffers(self):
        for b, init in zip(self.dbufs, self.prog.buf_init):
            if init.size:
                b.copy_(self.torch.from_numpy(np.ascontiguousarray(init)).to(b.device))
        self.st.zero_()
        self.torch.cuda.synchronize()

    def errors(self):
        mpx = self.mpx
        return [mpx.mpx_stream_get_error(s) for s in self.ms], mpx.mpx_world_get_error(self.world)

    def close(self):
        mpx = self.mpx
        if self.graph:
            if not self.finish():
                mpx.mpx_world_abort(self.world)
                t1 = time.perf_counter()
                while time.perf_counter() - t1 < 10 and not self.engine_stream.query():
                    time.sleep(1e-3)
            mpx.mpx_step_free(self.step_handle)
            self.graph = False
        if not self.finish():
            mpx.mpx_world_abort(self.world)
            t1 = time.perf_counter()
            while time.perf_counter() - t1 < 10 and not all(s.query() for s in self.cstreams):
                time.sleep(1e-3)
        for cl in self.comms:
            for h in cl:
                mpx.mpx_comm_free(h)
        for s in self.ms:
            for _ in range(2000):
                try:
                    mpx.mpx_stream_free(s)
                    break
                except mpx.MpxError as e:
                    if e.code != mpx.ERR_PENDING:
                        raise
                    time.sleep(5e-4)
        mpx.mpx_world_free(self.world)
        for h in self.raw:
            mpx.mpx_cuda_stream_destroy(h)
        for t in self.tmap[5:]:
            mpx.mpx_type_free(int(t))


def run_recorded_allreduce(prog: Program, timeout_s: float = 60.0) -> GpuOutcome:
    """A program whose streams hold only blocking allreduces in the comm's
    reduce mode, run as one recorded step (drain-mode world, exclusive
    streams): one CUDA graph of the descriptor publication kernel and one
    engine pass, launched on the engine stream.  No user stream waits on
    anything, so a kernel-serialising profiler can replay every launch."""
    import torch
    from paper_2208_13707_gb300 import mpx
    assert np.all(prog.ops["kind"] == ALLREDUCE), "allreduce-only programs"
    dev = torch.device("cuda")
    cfg = make_config(prog, mpx.ENGINE_DRAIN)
    dbufs = [torch.from_numpy(np.ascontiguousarray(b)).to(dev) if b.size else
             torch.empty(16, dtype=torch.uint8, device=dev) for b in prog.buf_init]
    torch.cuda.current_stream(dev).synchronize()
    ptr = [b.data_ptr() for b in dbufs]
    world = mpx.mpx_world_create(prog.nranks, cfg)
    raw = [mpx.mpx_cuda_stream_create() for _ in range(prog.nstreams + 1)]
    ms = [mpx.mpx_stream_create(world, int(prog.stream_rank[g]), raw[g], mpx.STREAM_EXCLUSIVE)
          for g in range(prog.nstreams)]
    comms = [mpx.mpx_stream_comm_create(world, [ms[int(g)] for g in prog.comm_stream[c]])
             for c in range(prog.ncomms)]
    rank_in = {(c, int(g)): r for c in range(prog.ncomms) for r, g in enumerate(prog.comm_stream[c])}
    ops = np.zeros(len(prog.ops), mpx.op_dtype())
    for j, o in enumerate(prog.ops):
        c, g = int(o["comm"]), int(o["stream"])
        ops[j]["kind"] = mpx.OP_ALLREDUCE
        ops[j]["datatype"] = int(o["type"])
        ops[j]["count"] = int(o["count"])
        ops[j]["op"] = mpx.SUM
        ops[j]["buf"] = mpx.IN_PLACE if int(o["buf"]) == IN_PLACE else ptr[int(o["buf"])] + int(o["off"])
        ops[j]["recvbuf"] = ptr[int(o["buf2"])] + int(o["off2"])
        ops[j]["comm"] = comms[c][rank_in[(c, g)]]
    t0 = time.perf_counter()
    step = mpx.mpx_step_create(world, ops)
    es = torch.cuda.ExternalStream(raw[-1], device=dev)
    mpx.mpx_step_launch(step, raw[-1])
    finished = False
    while time.perf_counter() - t0 < timeout_s:
        if es.query():
            finished = True
            break
        time.sleep(1e-4)
    if not finished:
        mpx.mpx_world_abort(world)
        t1 = time.perf_counter()
        while time.perf_counter() - t1 < 10 and not es.query():
            time.sleep(1e-3)
    out = [b.cpu().numpy()[: prog.buf_init[i].size].copy() for i, b in enumerate(dbufs)] if finished else []
    werr = mpx.mpx_world_get_error(world)
    serr = [mpx.mpx_step_get_error(step)]
    counters = mpx.mpx_world_get_counters(world)
    mpx.mpx_step_free(step)
    if finished:
        for cl in comms:
            for h in cl:
                mpx.mpx_comm_free(h)
        for s in ms:
            mpx.mpx_stream_free(s)
        mpx.mpx_world_free(world)
        for h in raw:
            mpx.mpx_cuda_stream_destroy(h)
    return GpuOutcome(buffers=out, status=np.zeros(0, STATUS_DTYPE), stream_errors=serr, world_error=werr,
                      counters=counters, finished=finished, seconds=time.perf_counter() - t0)
