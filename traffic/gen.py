"""Seeded synthetic workloads, one builder per traffic shape.

Every workload is a closed `Program` (see program.py).  Only random draws and
layout bookkeeping live here; how operations match, what bytes land where and
what a reduction yields is left to the code under test and to the oracle.
Seeds follow the convention seed = 0x220813707 + workload index.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence

import numpy as np

from .program import (ANY_INDEX, ANY_SOURCE, ANY_TAG, IALLREDUCE, IBCAST, IN_PLACE, MODE_FIXED,
                      MODE_TREE, T_BYTE, T_DOUBLE, T_FLOAT, T_INT32, T_INT64, BASIC_SIZES, Program,
                      ProgramBuilder)
from .rng import Rng

SEED_BASE = 0x220813707


# ----------------------------------------------------------------------------
# Worked examples of §6
# ----------------------------------------------------------------------------
def listing4(n: int = 1 << 20, a: float = 2.0, x_val: float = 1.0, y_val: float = 2.0) -> Program:
    """Listing 4 (§6): rank 0 sends x (all x_val) to rank 1, which receives it
    into device memory and runs y = a*x + y in stream order.  With the printed
    constants every y[i] ends as 2*1+2 = 4."""
    b = ProgramBuilder(2, "listing4")
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    x = b.buffer(np.full(n, x_val, np.float32))
    dx = b.buffer(4 * n)
    dy = b.buffer(np.full(n, y_val, np.float32))
    b.send(g0, c, x, 0, n, T_FLOAT, 1, 0)
    b.recv(g1, c, dx, 0, n, T_FLOAT, 0, 0)
    b.axpy(g1, a, dx, 0, dy, 0, n)
    b.meta.update(x=x, dx=dx, dy=dy, n=n)
    return b.build()


def listing3(nt: int = 4, nbytes: int = 100, seed: int = SEED_BASE) -> Program:
    """Listing 3 (§6): NT streams per rank, one stream communicator per thread
    index; thread i of rank 0 sends 100 chars to thread i of rank 1 (tag 0)."""
    b = ProgramBuilder(2, "listing3")
    s0 = [b.stream(0) for _ in range(nt)]
    s1 = [b.stream(1) for _ in range(nt)]
    comms = [b.comm([s0[i], s1[i]]) for i in range(nt)]
    rng = Rng(seed, 3)
    src = [b.buffer(rng.bytes(nbytes)) for _ in range(nt)]
    dst = [b.buffer(nbytes) for _ in range(nt)]
    for i in range(nt):
        b.send(s0[i], comms[i], src[i], 0, nbytes, T_BYTE, 1, 0)
        b.recv(s1[i], comms[i], dst[i], 0, nbytes, T_BYTE, 0, 0)
    b.meta.update(src=src, dst=dst)
    return b.build()


# ----------------------------------------------------------------------------
# Tiny instance: 2 ranks, blocking sends and permuted blocking receives
# ----------------------------------------------------------------------------
def tiny_pairs(nmsg: int = 1000, max_count: int = 4096, ntags: int = 8,
               seed: int = SEED_BASE + 0) -> Program:
    """2 virtual ranks, one stream each.  Rank 0 issues `nmsg` blocking sends of
    int32 payloads (count ~ U[1, max_count], tag ~ U[0, ntags-1]); rank 1 issues
    blocking receives in a seeded permutation that keeps the per-tag order, each
    with exactly the matching message's count."""
    rng = Rng(seed, 1)
    counts = rng.integers(1, max_count, nmsg)
    tags = rng.integers(0, ntags - 1, nmsg)
    # a uniformly random interleaving of the per-tag subsequences
    order = rng.permutation(nmsg)
    recv_order = np.empty(nmsg, np.int64)
    slots_by_tag = {}
    for pos, m in enumerate(order):
        slots_by_tag.setdefault(int(tags[m]), []).append(pos)
    for t, slots in slots_by_tag.items():
        msgs = np.nonzero(tags == t)[0]
        recv_order[np.array(slots)] = msgs
    offs = np.concatenate([[0], np.cumsum(counts * 4)])
    total = int(offs[-1])
    b = ProgramBuilder(2, "tiny_pairs")
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    sbuf = b.buffer(rng.integers(-(1 << 31), (1 << 31) - 1, total // 4).astype(np.int32))
    rbuf = b.buffer(total)
    st = b.status_slots(nmsg)
    for m in range(nmsg):
        b.send(g0, c, sbuf, int(offs[m]), int(counts[m]), T_INT32, 1, int(tags[m]))
    for i, m in enumerate(recv_order):
        b.recv(g1, c, rbuf, int(offs[m]), int(counts[m]), T_INT32, 0, int(tags[m]), st + i)
    b.meta.update(counts=counts, tags=tags, recv_order=recv_order, sbuf=sbuf, rbuf=rbuf,
                  payload_bytes=total, nmsg=nmsg)
    return b.build()


# ----------------------------------------------------------------------------
# Ring exchange interleaved with an axpy per step
# ----------------------------------------------------------------------------
def _ring_message(seed: int, step: int, rank: int, direction: int,
                  min_bytes: int, max_bytes: int):
    """Size and layout of the message `rank` sends in `direction` (0: to rank+1,
    1: to rank-1) at `step`.  Both ends derive it from the same key.
    layout: 0 contig->contig, 1 vector->vector, 2 vector->contig, 3 contig->vector."""
    r = Rng(seed, 2, step, rank, direction)
    nbytes = float(r.log_uniform(min_bytes, max_bytes, 1)[0])
    layout = int(r.integers(0, 3, 1)[0])
    if layout == 0:
        nbytes = max(4, int(nbytes) // 4 * 4)
    else:
        nbytes = max(256, int(nbytes) // 256 * 256)
    return nbytes, layout


def ring_exchange(nranks: int = 8, n: int = 1 << 24, steps: int = 200,
                  min_bytes: int = 4096, max_bytes: int = 64 << 20,
                  alpha: float = 0.5, seed: int = SEED_BASE + 1,
                  blocklen: int = 64, stride: int = 128) -> Program:
    """R ranks in a ring, one stream each.  Per step on every rank: an fp32
    axpy y = alpha*x + y over n elements, isends to both neighbours, irecvs from
    both, then one waitall.  y is the head of the send arena S, x is the head of
    the receive arena RL (data from the left neighbour), so each step's sends
    carry the previous axpy's output and each axpy consumes the last message
    from the left.  Messages are fp32, log-uniform in bytes; half are sent as
    MPI_Type_vector(nb, blocklen, stride) and receive datatypes are either the
    same vector or contiguous (and vice versa)."""
    assert nranks >= 3
    arena = max(2 * max_bytes, 4 * n) + 4096
    b = ProgramBuilder(nranks, "ring_exchange")
    gs = [b.stream(r) for r in range(nranks)]
    c = b.comm(gs)
    S, RL, RR = [], [], []
    for r in range(nranks):
        rng = Rng(seed, 20, r)
        s_init = np.zeros(arena // 4, np.float32)
        s_init[:] = rng.normal(arena // 4).astype(np.float32)
        S.append(b.buffer(s_init))
        x_init = np.zeros(arena // 4, np.float32)
        x_init[:] = rng.normal(arena // 4).astype(np.float32)
        RL.append(b.buffer(x_init))
        RR.append(b.buffer(arena))
    vtypes = {}

    def vtype(nb):
        if nb not in vtypes:
            vtypes[nb] = b.vector(nb, blocklen, stride, T_FLOAT)
        return vtypes[nb]

    def send_layout(nbytes, layout):
        if layout in (1, 2):
            return 1, vtype(nbytes // (4 * blocklen))
        return nbytes // 4, T_FLOAT

    def recv_layout(nbytes, layout):
        if layout in (1, 3):
            return 1, vtype(nbytes // (4 * blocklen))
        return nbytes // 4, T_FLOAT

    total_payload = 0
    for step in range(steps):
        for r in range(nranks):
            g = gs[r]
            right, left = (r + 1) % nranks, (r - 1) % nranks
            b.axpy(g, alpha, RL[r], 0, S[r], 0, n)
            reqs = []
            for direction, dest in ((0, right), (1, left)):
                nbytes, layout = _ring_message(seed, step, r, direction, min_bytes, max_bytes)
                cnt, ty = send_layout(nbytes, layout)
                reqs.append(b.isend(g, c, S[r], 0, cnt, ty, dest, direction))
                total_payload += nbytes
            # receive from left the message it sent rightwards (tag 0), and from
            # right the message it sent leftwards (tag 1)
            for direction, src, dstbuf in ((0, left, RL[r]), (1, right, RR[r])):
                nbytes, layout = _ring_message(seed, step, src, direction, min_bytes, max_bytes)
                cnt, ty = recv_layout(nbytes, layout)
                reqs.append(b.irecv(g, c, dstbuf, 0, cnt, ty, src, direction))
            b.waitall(g, reqs)
    b.meta.update(S=S, RL=RL, RR=RR, n=n, steps=steps, payload_bytes=total_payload,
                  messages=2 * nranks * steps, alpha=alpha)
    return b.build()


# ----------------------------------------------------------------------------
# Enqueued allreduce over R ranks
# ----------------------------------------------------------------------------
def allreduce_suite(nranks: int = 16, sizes: Sequence[int] = (1024,),
                    dtypes: Sequence[int] = (T_INT64, T_FLOAT),
                    modes: Sequence[int] = (MODE_FIXED, MODE_TREE),
                    in_place: bool = False, seed: int = SEED_BASE + 3) -> Program:
    """Every rank's single stream runs one allreduce(SUM) per (size, dtype,
    mode) in the same order.  int64 values are round(N(0,1)*2^40); fp32/fp64
    values are N(0,1); int32 values are uniform over the full range."""
    b = ProgramBuilder(nranks, "allreduce")
    gs = [b.stream(r) for r in range(nranks)]
    c = b.comm(gs)
    inst = []
    k = 0
    for n in sizes:
        for dt in dtypes:
            modes_here = modes if dt in (T_FLOAT, T_DOUBLE) else (MODE_FIXED,)
            for mode in modes_here:
                sb, rb = [], []
                for r in range(nranks):
                    rng = Rng(seed, 30, k, r)
                    if dt == T_INT64:
                        v = np.rint(rng.normal(n) * float(1 << 40)).astype(np.int64)
                    elif dt == T_FLOAT:
                        v = rng.normal(n).astype(np.float32)
                    elif dt == T_DOUBLE:
                        v = rng.normal(n)
                    elif dt == T_INT32:
                        v = rng.integers(-(1 << 31), (1 << 31) - 1, n).astype(np.int32)
                    else:
                        v = rng.bytes(n)
                    if in_place:
                        rb.append(b.buffer(v))
                        sb.append(IN_PLACE)
                    else:
                        sb.append(b.buffer(v))
                        rb.append(b.buffer(n * BASIC_SIZES[dt]))
                for r in range(nranks):
                    b.allreduce(gs[r], c, sb[r], 0, rb[r], 0, n, dt, mode)
                inst.append(dict(n=n, dtype=dt, mode=mode, send=sb, recv=rb))
                k += 1
    b.meta.update(instances=inst)
    return b.build()


# ----------------------------------------------------------------------------
# 3-D 7-point halo exchange on a periodic 2x2x2 decomposition
# ----------------------------------------------------------------------------
def halo3d(sub: int = 256, steps: int = 100, seed: int = SEED_BASE + 3, init: bool = True) -> Program:
    """A (2*sub)^3 fp32 grid split into 8 subdomains of sub^3 ([z][y][x]), one
    rank and one stream each, periodic boundaries.  Per step each rank sends its
    6 boundary faces (x faces as vector(sub*sub, 1, sub), y faces as
    vector(sub, sub, sub*sub), z faces contiguous) to the neighbour across that
    face (tag = face id), receives 6 faces into 6 contiguous ghost buffers, and
    waits for all 12 requests.  init=False leaves the subdomains zero (for
    callers that fill them on the device)."""
    nr = 8
    b = ProgramBuilder(nr, "halo3d")
    gs = [b.stream(r) for r in range(nr)]
    c = b.comm(gs)
    plane = sub * sub
    tx = b.vector(plane, 1, sub, T_FLOAT)
    ty = b.vector(sub, sub, plane, T_FLOAT)
    U, G = [], []
    for r in range(nr):
        U.append(b.buffer(Rng(seed, 40, r).normal(sub ** 3).astype(np.float32) if init
                          else 4 * sub ** 3))
        G.append([b.buffer(4 * plane) for _ in range(6)])

    def coords(r):
        return r & 1, (r >> 1) & 1, (r >> 2) & 1

    def rank_of(px, py, pz):
        return (px % 2) | ((py % 2) << 1) | ((pz % 2) << 2)

    # face f: 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+ ; (type, count, byte offset)
    faces = [(tx, 1, 0), (tx, 1, 4 * (sub - 1)),
             (ty, 1, 0), (ty, 1, 4 * sub * (sub - 1)),
             (T_FLOAT, plane, 0), (T_FLOAT, plane, 4 * plane * (sub - 1))]
    shift = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    for step in range(steps):
        for r in range(nr):
            px, py, pz = coords(r)
            reqs = []
            for f in range(6):
                dx, dy, dz = shift[f]
                dest = rank_of(px + dx, py + dy, pz + dz)
                t, cnt, off = faces[f]
                reqs.append(b.isend(gs[r], c, U[r], off, cnt, t, dest, f))
            for f in range(6):
                # the ghost for face f is the opposite face of the neighbour across f
                dx, dy, dz = shift[f]
                src = rank_of(px + dx, py + dy, pz + dz)
                opposite = f ^ 1
                reqs.append(b.irecv(gs[r], c, G[r][f], 0, plane, T_FLOAT, src, opposite))
            b.waitall(gs[r], reqs)
    b.meta.update(U=U, G=G, sub=sub, steps=steps, payload_bytes=steps * nr * 6 * 4 * plane,
                  messages=steps * nr * 6)
    return b.build()


# ----------------------------------------------------------------------------
# Many ranks x several streams, random sizes, wildcard receives
# ----------------------------------------------------------------------------
def batching(nranks: int = 64, streams_per_rank: int = 4, nmsg: int = 1_000_000,
             min_bytes: int = 8, max_bytes: int = 1 << 20, ntags: int = 32,
             p_any_tag: float = 0.05, p_any_source: float = 0.02,
             seed: int = SEED_BASE + 2,
             fixup: Optional[Callable[[Program], Optional[np.ndarray]]] = None,
             max_fixups: int = 8, laminar: bool = False) -> Program:
    """R ranks x S streams; stream comm c holds every rank's c-th stream.  Each
    message has a uniform source stream, a uniform destination rank (same comm
    index), a uniform tag and log-uniform bytes; its dtype is uniform over
    {uint8, int32, fp32}.  Every stream isends and irecvs everything it owns in
    one seeded order and ends with one waitall.  In every (comm, destination)
    domain exact receives come before wildcard ones.  A receive is ANY_TAG with
    p_any_tag and ANY_SOURCE with p_any_source; wildcard receives get the
    maximum capacity of the messages they may take.

    `fixup`, when given, receives the program and returns the receive op
    indices that can never match (or None); those receives are widened to
    (ANY_SOURCE, ANY_TAG) and the program is rebuilt, up to `max_fixups` times.

    `laminar` makes every program complete without that check: an ANY_SOURCE
    receive is also ANY_TAG, so a domain's receive patterns are exact (s, t),
    (s, ANY_TAG) or (ANY_SOURCE, ANY_TAG) and any two are nested or disjoint.
    Posted most specific first, greedy matching in post-key order then never
    strands a receive.  Every receive gets the largest capacity among the
    messages its pattern admits, so none truncates either."""
    rng = Rng(seed, 50)
    ns = nranks * streams_per_rank
    src_stream = rng.integers(0, ns - 1, nmsg)
    dst_rank = rng.integers(0, nranks - 1, nmsg)
    tags = rng.integers(0, ntags - 1, nmsg)
    nbytes_f = rng.log_uniform(min_bytes, max_bytes, nmsg)
    dt_choice = rng.integers(0, 2, nmsg)
    dts = np.array([T_BYTE, T_INT32, T_FLOAT])[dt_choice]
    esz = np.array([1, 4, 4])[dt_choice]
    counts = np.maximum(1, nbytes_f.astype(np.int64) // esz)
    wild_tag = rng.uniform(nmsg) < p_any_tag
    wild_src = rng.uniform(nmsg) < p_any_source
    send_key = rng.u64(nmsg)
    recv_key = rng.u64(nmsg)
    widened = np.zeros(nmsg, bool)
    if laminar:
        wild_tag = wild_tag | wild_src
    for attempt in range(max_fixups + 1):
        prog = _batching_build(nranks, streams_per_rank, src_stream, dst_rank, tags,
                               counts, dts, esz, wild_tag | widened, wild_src | widened,
                               send_key, recv_key, seed, laminar)
        if fixup is None:
            break
        bad = fixup(prog)
        if bad is None or len(bad) == 0:
            break
        msg_of_recv = prog.meta["msg_of_op"]
        for op in bad:
            m = msg_of_recv.get(int(op))
            if m is not None:
                widened[m] = True
    prog.meta["widened"] = int(widened.sum())
    return prog


def _batching_build(nranks, spr, src_stream, dst_rank, tags, counts, dts, esz,
                    wild_tag, wild_src, send_key, recv_key, seed, laminar=False) -> Program:
    nmsg = len(src_stream)
    ns = nranks * spr
    b = ProgramBuilder(nranks, "batching")
    gid = {}
    for r in range(nranks):
        for s in range(spr):
            gid[(r, s)] = b.stream(r)
    comms = [b.comm([gid[(r, s)] for r in range(nranks)]) for s in range(spr)]
    src_rank = src_stream // spr
    comm_of = src_stream % spr
    dst_stream = dst_rank * spr + comm_of
    nbytes = counts * esz
    # capacity of a wildcard receive: the largest message it could take
    cap = nbytes.copy()
    dom = comm_of * nranks + dst_rank
    maxdom = np.zeros(spr * nranks, np.int64)
    np.maximum.at(maxdom, dom, nbytes)
    wild = wild_tag | wild_src
    cap[wild] = maxdom[dom[wild]]
    if laminar:
        # (s, ANY_TAG): largest message from s in the domain; exact (s, t):
        # largest (s, t) message, since a wildcard may take an earlier one
        src_rank_ = src_stream // spr
        key_s = dom * nranks + src_rank_
        max_s = np.zeros(spr * nranks * nranks, np.int64)
        np.maximum.at(max_s, key_s, nbytes)
        key_st = key_s * (int(tags.max()) + 1) + tags
        uniq, inv = np.unique(key_st, return_inverse=True)
        max_st = np.zeros(len(uniq), np.int64)
        np.maximum.at(max_st, inv, nbytes)
        only_tag = wild_tag & ~wild_src
        cap = max_st[inv].copy()
        cap[only_tag] = max_s[key_s[only_tag]]
        cap[wild_src] = maxdom[dom[wild_src]]
        cap = (np.maximum(cap, esz) + esz - 1) // esz * esz
    # per-stream send arenas (payload) and receive arenas (capacity)
    send_off = np.zeros(nmsg, np.int64)
    recv_off = np.zeros(nmsg, np.int64)
    send_tot = np.zeros(ns, np.int64)
    recv_tot = np.zeros(ns, np.int64)
    for m in range(nmsg):
        gs_, gd = int(src_stream[m]), int(dst_stream[m])
        send_off[m] = send_tot[gs_]
        send_tot[gs_] += (nbytes[m] + 15) // 16 * 16
        recv_off[m] = recv_tot[gd]
        recv_tot[gd] += (cap[m] + 15) // 16 * 16
    sbufs = []
    for g in range(ns):
        sbufs.append(b.buffer(Rng(seed, 51, g).bytes(int(send_tot[g]))))
    rbufs = [b.buffer(int(recv_tot[g])) for g in range(ns)]
    # order: per stream, all of its sends and receives in a seeded order, except
    # that within a destination domain exact receives precede wildcard ones
    per_stream_items = [[] for _ in range(ns)]
    for m in range(nmsg):
        per_stream_items[int(src_stream[m])].append((int(send_key[m]), 0, m))
        rk = int(recv_key[m])
        level = int(wild_tag[m]) + 2 * int(wild_src[m])
        per_stream_items[int(dst_stream[m])].append((rk, 1 + level, m))
    msg_of_op = {}
    status_base = {}
    for g in range(ns):
        items = per_stream_items[g]
        sends = [it for it in items if it[1] == 0]
        recvs = [it for it in items if it[1] > 0]
        recvs.sort(key=lambda it: (it[1], it[0]))    # exact < ANY_TAG < ANY_SOURCE < both
        sends.sort(key=lambda it: it[0])
        # interleave sends and the (level-ordered) receives by their keys' ranks
        merged = []
        i = j = 0
        while i < len(sends) or j < len(recvs):
            take_send = j >= len(recvs) or (i < len(sends) and sends[i][0] < recvs[j][0])
            if take_send:
                merged.append(sends[i]); i += 1
            else:
                merged.append(recvs[j]); j += 1
        reqs = []
        for key, kind, m in merged:
            r = g // spr
            c = comms[g % spr]
            if kind == 0:
                h = b.isend(g, c, sbufs[g], int(send_off[m]), int(counts[m]), int(dts[m]),
                            int(dst_rank[m]), int(tags[m]))
            else:
                source = ANY_SOURCE if wild_src[m] else int(src_rank[m])
                tag = ANY_TAG if wild_tag[m] else int(tags[m])
                h = b.irecv(g, c, rbufs[g], int(recv_off[m]), int(cap[m] // esz[m]),
                            int(dts[m]), source, tag)
            reqs.append(h)
        if reqs:
            sb = b.status_slots(len(reqs))
            status_base[g] = sb
            b.waitall(g, reqs, sb)
    prog = b.build()
    # map receive op index -> message id by walking each stream in order
    lo = prog.stream_op_lo
    for g in range(ns):
        items = per_stream_items[g]
        sends = sorted([it for it in items if it[1] == 0], key=lambda it: it[0])
        recvs = sorted([it for it in items if it[1] > 0], key=lambda it: (it[1], it[0]))
        i = j = 0
        k = int(lo[g])
        while i < len(sends) or j < len(recvs):
            take_send = j >= len(recvs) or (i < len(sends) and sends[i][0] < recvs[j][0])
            if take_send:
                i += 1
            else:
                msg_of_op[k] = recvs[j][2]; j += 1
            k += 1
    prog.meta.update(msg_of_op=msg_of_op, payload_bytes=int(nbytes.sum()), messages=nmsg,
                     nbytes=nbytes, src_stream=src_stream, dst_stream=dst_stream)
    return prog


# ----------------------------------------------------------------------------
# Small random programs for exhaustive checks
# ----------------------------------------------------------------------------
def random_small(seed: int, nranks: int = 3, nmsg: int = 5, p_any_src: float = 0.3,
                 p_any_tag: float = 0.3, ntags: int = 2, p_blocking: float = 0.4,
                 max_count: int = 4) -> Program:
    """A handful of messages among `nranks` single-stream ranks with a mix of
    blocking and nonblocking calls, waits at random later points, and
    wildcard receives.  Receive capacities are the maximum message size, so
    every match delivers the whole message."""
    rng = Rng(seed, 60)
    b = ProgramBuilder(nranks, "random_small")
    gs = [b.stream(r) for r in range(nranks)]
    c = b.comm(gs)
    src = rng.integers(0, nranks - 1, nmsg)
    dst = rng.integers(0, nranks - 1, nmsg)
    tags = rng.integers(0, ntags - 1, nmsg)
    cnts = rng.integers(1, max_count, nmsg)
    anys = rng.uniform(nmsg) < p_any_src
    anyt = rng.uniform(nmsg) < p_any_tag
    sbuf = [b.buffer(rng.bytes(4 * max_count * nmsg)) for _ in range(nranks)]
    rbuf = [b.buffer(4 * max_count * nmsg) for _ in range(nranks)]
    items = [[] for _ in range(nranks)]
    keys = rng.uniform(2 * nmsg)
    blocking = rng.uniform(2 * nmsg) < p_blocking
    for m in range(nmsg):
        items[int(src[m])].append((keys[2 * m], "s", m, bool(blocking[2 * m])))
        items[int(dst[m])].append((keys[2 * m + 1], "r", m, bool(blocking[2 * m + 1])))
    for r in range(nranks):
        its = sorted(items[r])
        pending = []
        for key, kind, m, blk in its:
            m = int(m)
            if kind == "s":
                if blk:
                    b.send(gs[r], c, sbuf[r], 4 * max_count * m, int(cnts[m]), T_INT32,
                           int(dst[m]), int(tags[m]))
                else:
                    pending.append(b.isend(gs[r], c, sbuf[r], 4 * max_count * m, int(cnts[m]),
                                           T_INT32, int(dst[m]), int(tags[m])))
            else:
                source = ANY_SOURCE if anys[m] else int(src[m])
                tag = ANY_TAG if anyt[m] else int(tags[m])
                if blk:
                    b.recv(gs[r], c, rbuf[r], 4 * max_count * m, max_count, T_INT32,
                           source, tag, b.status_slots(1))
                else:
                    pending.append(b.irecv(gs[r], c, rbuf[r], 4 * max_count * m, max_count,
                                           T_INT32, source, tag))
            # occasionally complete some pending requests
            if pending and float(rng.uniform(1)[0]) < 0.35:
                k = int(rng.integers(1, len(pending), 1)[0])
                chosen, pending = pending[:k], pending[k:]
                if len(chosen) == 1:
                    b.wait(gs[r], chosen[0], b.status_slots(1))
                else:
                    b.waitall(gs[r], chosen, b.status_slots(len(chosen)))
        if pending:
            b.waitall(gs[r], pending, b.status_slots(len(pending)))
    return b.build()


# ----------------------------------------------------------------------------
# Multiplex stream communicators (§3.5)
# ----------------------------------------------------------------------------
def multiplex_small(seed: int, nranks: int = 2, counts: Sequence[int] = (2, 3), nmsg: int = 6,
                    p_any_src: float = 0.3, p_any_idx: float = 0.3, p_any_tag: float = 0.3,
                    ntags: int = 2, p_blocking: float = 0.3, max_count: int = 4,
                    p_wait: float = 0.35) -> Program:
    """A handful of messages between the (rank, local index) members of one
    multiplex stream communicator: rank r attaches counts[r] streams.  Sends
    name the destination's stream; receives name the source rank and index,
    either of which may be a wildcard, and the tag.  Blocking and nonblocking
    calls mix as in `random_small` (a waitall over some pending requests
    follows a call with probability p_wait); capacities are the largest
    message."""
    assert len(counts) == nranks
    rng = Rng(seed, 61)
    b = ProgramBuilder(nranks, "multiplex_small")
    local = [[b.stream(r) for _ in range(int(counts[r]))] for r in range(nranks)]
    c = b.comm_multiple(local)
    members = [(r, i) for r in range(nranks) for i in range(int(counts[r]))]
    src = rng.integers(0, len(members) - 1, nmsg)
    dst = rng.integers(0, len(members) - 1, nmsg)
    tags = rng.integers(0, ntags - 1, nmsg)
    cnts = rng.integers(1, max_count, nmsg)
    anys = rng.uniform(nmsg) < p_any_src
    anyi = rng.uniform(nmsg) < p_any_idx
    anyt = rng.uniform(nmsg) < p_any_tag
    keys = rng.uniform(2 * nmsg)
    blocking = rng.uniform(2 * nmsg) < p_blocking
    sbuf = {m: b.buffer(rng.bytes(4 * max_count * nmsg)) for m in members}
    rbuf = {m: b.buffer(4 * max_count * nmsg) for m in members}
    items = {m: [] for m in members}
    for k in range(nmsg):
        items[members[int(src[k])]].append((keys[2 * k], "s", k, bool(blocking[2 * k])))
        items[members[int(dst[k])]].append((keys[2 * k + 1], "r", k, bool(blocking[2 * k + 1])))
    for m in members:
        g = local[m[0]][m[1]]
        pending = []
        for key, kind, k, blk in sorted(items[m]):
            k = int(k)
            off = 4 * max_count * k
            if kind == "s":
                dr, di = members[int(dst[k])]
                h = b.stream_send(g, c, sbuf[m], off, int(cnts[k]), T_INT32, dr, di, int(tags[k]),
                                  blocking=blk)
            else:
                sr, si = members[int(src[k])]
                h = b.stream_recv(g, c, rbuf[m], off, max_count, T_INT32,
                                  ANY_SOURCE if anys[k] else sr, ANY_INDEX if anyi[k] else si,
                                  ANY_TAG if anyt[k] else int(tags[k]), blocking=blk,
                                  status=b.status_slots(1) if blk else -1)
            if not blk:
                pending.append(h)
            if pending and float(rng.uniform(1)[0]) < p_wait:
                n = int(rng.integers(1, len(pending), 1)[0])
                chosen, pending = pending[:n], pending[n:]
                b.waitall(g, chosen, b.status_slots(len(chosen)))
        if pending:
            b.waitall(g, pending, b.status_slots(len(pending)))
    return b.build()


def n_to_one(nranks: int = 4, threads: int = 4, msgs: int = 8, max_bytes: int = 4096,
             seed: int = SEED_BASE + 5) -> Program:
    """The N-to-1 pattern of §3.5: every rank attaches `threads` streams to
    one multiplex stream communicator; every stream except rank 0's stream 0
    sends `msgs` messages to that polling stream, whose receives are all
    (ANY_SOURCE, ANY_INDEX, ANY_TAG).  Message k of sender (r, i) has tag k
    and log-uniform size (bytes of int32 elements); every receive has the
    largest capacity.  Each sender ends with a waitall, the poller with one
    waitall over all its receives (statuses recorded)."""
    rng = Rng(seed, 62)
    b = ProgramBuilder(nranks, "n_to_one")
    local = [[b.stream(r) for _ in range(threads)] for r in range(nranks)]
    c = b.comm_multiple(local)
    senders = [(r, i) for r in range(nranks) for i in range(threads) if (r, i) != (0, 0)]
    maxc = max(1, max_bytes // 4)
    nrecv = len(senders) * msgs
    rb = b.buffer(4 * maxc * nrecv)
    for (r, i) in senders:
        sizes = np.maximum(1, np.exp(rng.uniform(msgs) * np.log(maxc)).astype(np.int64))
        sb = b.buffer(rng.bytes(4 * maxc * msgs))
        g = local[r][i]
        reqs = [b.stream_send(g, c, sb, 4 * maxc * k, int(sizes[k]), T_INT32, 0, 0, k)
                for k in range(msgs)]
        b.waitall(g, reqs)
    poll = local[0][0]
    reqs = [b.stream_recv(poll, c, rb, 4 * maxc * q, maxc, T_INT32, ANY_SOURCE, ANY_INDEX, ANY_TAG)
            for q in range(nrecv)]
    b.waitall(poll, reqs, b.status_slots(nrecv))
    return b.build()


# ----------------------------------------------------------------------------
# Serving: open-loop requests of many host threads (reading A12)
# ----------------------------------------------------------------------------
SERVE_SEND, SERVE_RECV, SERVE_WAITALL, SERVE_ALLREDUCE = 0, 1, 2, 3
SERVE_CALL_DTYPE = np.dtype([("kind", "<i4"), ("peer", "<i4"), ("tag", "<i4"), ("pad", "<i4"),
                             ("item", "<i8"), ("bytes", "<i8"), ("off", "<i8"), ("capture", "<i8")])


def serving_schedule(nthreads: int = 8, requests: int = 2000, p_allreduce: float = 0.3,
                     min_log2: int = 6, max_log2: int = 14, zipf_s: float = 1.2,
                     seed: int = SEED_BASE + 4, only_items: Optional[Sequence[int]] = None) -> dict:
    """The serving workload as explicit per-thread call lists: every thread
    makes requests/nthreads calls, a share p_allreduce of them fp32 SUM
    allreduce participations (the same instance list on every thread), the
    rest isends and irecvs of messages with a uniform source, a uniform other
    destination, Zipf(zipf_s) power-of-two sizes over 2^min_log2..2^max_log2
    and a tag counting the messages of their (source, destination) pair.  The
    calls between two allreduce instances form an epoch: each thread issues
    its sends and receives of the epoch in a seeded order, a waitall, then the
    epoch's allreduce.  Items: messages 0..M-1, then instances M..M+nar-1.

    Every receive and every thread's allreduce result gets its own slice of
    one capture area, and every waitall its own status slots, so a run's
    delivered bytes can be compared item by item.  `only_items` keeps just
    those items' calls (an item run alone).  Returns calls (SERVE_CALL_DTYPE,
    thread after thread), call_lo, regions (per thread fp32 N(0,1) data, as
    bytes), capture_bytes, nstatuses, and the item bookkeeping."""
    T = nthreads
    per = max(1, requests // T)
    nar = int(np.floor(p_allreduce * per + 0.5))
    M = (per - nar) * T // 2
    nb = max_log2 - min_log2 + 1
    w = 1.0 / np.arange(1, nb + 1, dtype=np.float64) ** zipf_s
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0

    def zipf(rng, n):
        k = np.searchsorted(cdf, rng.uniform(n), side="left")
        return np.left_shift(1, min_log2 + np.minimum(k, nb - 1)).astype(np.int64)

    maxb = 1 << max_log2
    region_bytes = 2 * maxb
    rm = Rng(seed, 70)
    src = rm.integers(0, T - 1, M)
    dst = rm.integers(0, T - 2, M)
    dst = dst + (dst >= src)
    epoch = rm.integers(0, nar, M)
    mbytes = zipf(rm, M)
    moff = (rm.integers(0, region_bytes, M) % (region_bytes - mbytes + 1)) & ~255
    tags = np.zeros(M, np.int64)
    pair = {}
    for m in range(M):
        k = (int(src[m]), int(dst[m]))
        tags[m] = pair.get(k, 0)
        pair[k] = tags[m] + 1
    ra = Rng(seed, 71)
    abytes = zipf(ra, nar) & ~3
    aoff = (ra.integers(0, region_bytes, nar) % (region_bytes - abytes + 1)) & ~255
    keep = None if only_items is None else set(int(i) for i in only_items)
    # capture slices: messages in item order, then each instance's T results
    cap_off = {}
    pos = 0
    for m in range(M):
        cap_off[m] = pos
        pos += (int(mbytes[m]) + 255) // 256 * 256
    for e in range(nar):
        for t in range(T):
            cap_off[(M + e, t)] = pos
            pos += (int(abytes[e]) + 255) // 256 * 256
    capture_bytes = max(pos, 256)
    ep = [[[] for _ in range(nar + 1)] for _ in range(T)]
    for m in range(M):
        if keep is not None and m not in keep:
            continue
        s_, d_, e_ = int(src[m]), int(dst[m]), int(epoch[m])
        ep[s_][e_].append((SERVE_SEND, d_, int(tags[m]), m, int(mbytes[m]), int(moff[m]), -1))
        ep[d_][e_].append((SERVE_RECV, s_, int(tags[m]), m, int(mbytes[m]), 0, cap_off[m]))
    rows, lo, nstat = [], [0], 0
    for t in range(T):
        rs = Rng(seed, 72, t)
        for e in range(nar + 1):
            v = ep[t][e]
            if v:
                order = rs.permutation(len(v))
                v = [v[int(i)] for i in order]
                rows.extend(v)
                n_req = len(v)
                rows.append((SERVE_WAITALL, 0, 0, 0, 0, 0, nstat))
                nstat += n_req
            if e < nar and (keep is None or M + e in keep):
                rows.append((SERVE_ALLREDUCE, 0, 0, M + e, int(abytes[e]), int(aoff[e]),
                             cap_off[(M + e, t)]))
        lo.append(len(rows))
    calls = np.zeros(len(rows), SERVE_CALL_DTYPE)
    for i, (k, peer, tag, item, b, off, cap) in enumerate(rows):
        calls[i] = (k, peer, tag, 0, item, b, off, cap)
    regions = [Rng(seed, 73, t).normal(region_bytes // 4).astype(np.float32).view(np.uint8)
               for t in range(T)]
    return dict(calls=calls, call_lo=np.array(lo, np.int64), regions=regions,
                region_bytes=region_bytes, capture_bytes=capture_bytes, nstatuses=max(nstat, 1),
                nthreads=T, messages=M, instances=nar, cap_off=cap_off, mbytes=mbytes, abytes=abytes)


def serving_program(sched: dict) -> Program:
    """The same calls as a closed program for the oracle: thread t is rank t
    with one stream; receives land in one capture buffer at their capture
    offsets, allreduce results too, waitall statuses in their slots."""
    T = sched["nthreads"]
    b = ProgramBuilder(T, "serving")
    gs = [b.stream(t) for t in range(T)]
    c = b.comm(gs)
    regs = [b.buffer(r) for r in sched["regions"]]
    cap = b.buffer(int(sched["capture_bytes"]))
    st0 = b.status_slots(int(sched["nstatuses"]))
    calls, lo = sched["calls"], sched["call_lo"]
    for t in range(T):
        reqs = []
        for x in calls[int(lo[t]): int(lo[t + 1])]:
            k = int(x["kind"])
            if k == SERVE_SEND:
                reqs.append(b.isend(gs[t], c, regs[t], int(x["off"]), int(x["bytes"]), T_BYTE,
                                    int(x["peer"]), int(x["tag"])))
            elif k == SERVE_RECV:
                reqs.append(b.irecv(gs[t], c, cap, int(x["capture"]), int(x["bytes"]), T_BYTE,
                                    int(x["peer"]), int(x["tag"])))
            elif k == SERVE_WAITALL:
                b.waitall(gs[t], reqs, st0 + int(x["capture"]))
                reqs = []
            else:
                b.allreduce(gs[t], c, regs[t], int(x["off"]), cap, int(x["capture"]),
                            int(x["bytes"]) // 4, T_FLOAT, MODE_FIXED)
    return b.build()


# ----------------------------------------------------------------------------
# Persistent collectives (MPI-4 MPI_Allreduce_init / MPI_Start in enqueue form)
# ----------------------------------------------------------------------------
def persistent_collectives(nranks: int = 4, starts: int = 3, n: int = 1000,
                           seed: int = SEED_BASE + 3) -> Program:
    """Every rank creates a persistent in-place int64 allreduce over Y and a
    persistent fp32 broadcast of B from root 1, then, `starts` times: starts
    the allreduce, waits, starts the broadcast, waits.  Between broadcast
    starts the root's B is rewritten by an axpy (B = 0.5 * X + B), so every
    start must read the buffer as it stands when the stream reaches it."""
    b = ProgramBuilder(nranks, "persistent")
    gs = [b.stream(r) for r in range(nranks)]
    c = b.comm(gs)
    Y, B, X = [], [], []
    for r in range(nranks):
        rng = Rng(seed, 80, r)
        Y.append(b.buffer(rng.integers(-(1 << 40), 1 << 40, n).astype(np.int64)))
        B.append(b.buffer(rng.normal(n).astype(np.float32)))
        X.append(b.buffer(rng.normal(n).astype(np.float32)))
    ar = [b.persistent(gs[r], IALLREDUCE, c, buf=IN_PLACE, off=0, buf2=Y[r], off2=0, count=n,
                       type=T_INT64, mode=MODE_FIXED) for r in range(nranks)]
    bc = [b.persistent(gs[r], IBCAST, c, buf=B[r], off=0, count=n, type=T_FLOAT, peer=1)
          for r in range(nranks)]
    for _ in range(starts):
        for r in range(nranks):
            b.wait(gs[r], b.start(gs[r], ar[r]))
            if r == 1:
                b.axpy(gs[r], 0.5, X[r], 0, B[r], 0, n)
            b.wait(gs[r], b.start(gs[r], bc[r]))
    b.meta.update(Y=Y, B=B, X=X, n=n, starts=starts)
    return b.build()
