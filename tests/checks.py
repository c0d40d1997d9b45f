"""Independent checks used to pin the oracle and to compare the GPU path.

Nothing here calls the oracle.  The helpers restate facts from MPI and the
MPIX Stream paper in forms different from the oracle's code:
  * `np_pack` / `np_unpack`: MPI_Type_vector as a column block of a 2-D array
    (reshape to (vcount, stride) rows, keep the first blocklen columns).
  * `closed_form_matches`: with no wildcards, the k-th send on
    (comm, src -> dst, tag) matches the k-th receive dst posts for
    (comm, src, tag) (§2.1: matching order is the outcome; non-overtaking).
    On a multiplex stream communicator (§3.5) src and dst are (rank, local
    stream index) pairs; a comm with one stream per rank has index 0 only.
  * `validity_violations`: necessary conditions any MPI-legal match map meets.
  * `legal_outcomes`: brute-force enumeration of every MPI-legal execution of a
    tiny program (arbitrary stream interleavings and per-channel FIFO message
    delays), giving the exact set of legal match maps.
"""
from __future__ import annotations

from collections import defaultdict
from typing import Dict, FrozenSet, List, Set, Tuple

import numpy as np

from traffic.program import (ALLREDUCE, ANY_INDEX, ANY_SOURCE, ANY_TAG, AXPY, ERR_TRUNCATE, IRECV,
                             ISEND, RECV, SEND, WAIT, WAITALL, Program)

SEND_KINDS = (SEND, ISEND)
RECV_KINDS = (RECV, IRECV)


def comm_rank(prog: Program, comm: int, g: int) -> int:
    m = prog.member(comm, g)
    return m[0] if m is not None else -1


def comm_member(prog: Program, comm: int, g: int) -> Tuple[int, int]:
    """(rank, local stream index) of stream g in comm (index 0 on a plain comm)."""
    m = prog.member(comm, g)
    return m if m is not None else (-1, -1)


# ---------------------------------------------------------------------------
# datatypes as 2-D array slices
# ---------------------------------------------------------------------------
def np_pack(buf: np.ndarray, off: int, types, t: int, count: int) -> np.ndarray:
    r = types[t]
    elem = int(r["elem"])
    if int(r["kind"]) == 0:
        return buf[off: off + count * elem].copy()
    vc, bl, st = int(r["vcount"]), int(r["blocklen"]), int(r["stride"])
    extent = ((vc - 1) * st + bl) * elem
    parts = []
    for i in range(count):
        base = off + i * extent
        rows = np.zeros(vc * st * elem, np.uint8)
        seg = buf[base: base + vc * st * elem]
        rows[: len(seg)] = seg
        parts.append(rows.reshape(vc, st * elem)[:, : bl * elem].reshape(-1))
    return np.concatenate(parts) if parts else np.zeros(0, np.uint8)


def np_unpack(buf: np.ndarray, off: int, types, t: int, count: int, data: np.ndarray) -> None:
    """Write the first len(data) bytes of the packed stream into buf."""
    r = types[t]
    elem = int(r["elem"])
    n = len(data)
    if int(r["kind"]) == 0:
        buf[off: off + n] = data
        return
    vc, bl, st = int(r["vcount"]), int(r["blocklen"]), int(r["stride"])
    extent = ((vc - 1) * st + bl) * elem
    per = vc * bl * elem
    done = 0
    for i in range(count):
        if done >= n:
            break
        base = off + i * extent
        take = min(per, n - done)
        avail = min(vc * st * elem, len(buf) - base)
        rows = np.zeros(vc * st * elem, np.uint8)
        rows[:avail] = buf[base: base + avail]
        view = rows.reshape(vc, st * elem)[:, : bl * elem].reshape(-1).copy()
        view[:take] = data[done: done + take]
        rows.reshape(vc, st * elem)[:, : bl * elem] = view.reshape(vc, bl * elem)
        buf[base: base + avail] = rows[:avail]
        done += take


# ---------------------------------------------------------------------------
# matching
# ---------------------------------------------------------------------------
def closed_form_matches(prog: Program) -> Dict[int, int]:
    """send op -> recv op for wildcard-free traffic."""
    sends = defaultdict(list)
    recvs = defaultdict(list)
    lo = prog.stream_op_lo
    for g in range(prog.nstreams):
        for j in range(int(lo[g]), int(lo[g + 1])):
            o = prog.ops[j]
            k = int(o["kind"])
            if k in SEND_KINDS:
                me = comm_member(prog, int(o["comm"]), g)
                dst = (int(o["peer"]), int(o["didx"]))
                sends[(int(o["comm"]), me, dst, int(o["tag"]))].append(j)
            elif k in RECV_KINDS:
                assert int(o["peer"]) != ANY_SOURCE and int(o["tag"]) != ANY_TAG
                assert int(o["sidx"]) != ANY_INDEX
                me = comm_member(prog, int(o["comm"]), g)
                src = (int(o["peer"]), int(o["sidx"]))
                recvs[(int(o["comm"]), src, me, int(o["tag"]))].append(j)
    out = {}
    for key, ss in sends.items():
        for s, r in zip(ss, recvs.get(key, [])):
            out[s] = r
    return out


def accepts(prog: Program, r: int, s: int) -> bool:
    ro, so = prog.ops[r], prog.ops[s]
    if int(ro["comm"]) != int(so["comm"]):
        return False
    if comm_member(prog, int(ro["comm"]), int(ro["stream"])) != (int(so["peer"]), int(so["didx"])):
        return False
    src, sidx = comm_member(prog, int(so["comm"]), int(so["stream"]))
    return (int(ro["peer"]) in (ANY_SOURCE, src)) and (int(ro["sidx"]) in (ANY_INDEX, sidx)) and \
        (int(ro["tag"]) in (ANY_TAG, int(so["tag"])))


def validity_violations(prog: Program, match: np.ndarray, require_complete: bool) -> List[str]:
    """Necessary conditions on a match map (match[op] = partner or -1)."""
    bad = []
    kinds = prog.ops["kind"]
    pairs = []
    for s in range(len(match)):
        if kinds[s] in SEND_KINDS and match[s] >= 0:
            r = int(match[s])
            if kinds[r] not in RECV_KINDS or int(match[r]) != s:
                bad.append(f"send {s} -> {r} not mutual")
                continue
            if not accepts(prog, r, s):
                bad.append(f"recv {r} cannot accept send {s}")
            pairs.append((s, r))
    for r in range(len(match)):
        if kinds[r] in RECV_KINDS:
            if match[r] >= 0 and (kinds[int(match[r])] not in SEND_KINDS or int(match[int(match[r])]) != r):
                bad.append(f"recv {r} partner not mutual")
            if require_complete and match[r] < 0:
                bad.append(f"recv {r} unmatched")
    # non-overtaking: same channel sends s1 < s2 matched to r1, r2 of one stream
    by_channel = defaultdict(list)
    for s, r in pairs:
        o = prog.ops[s]
        by_channel[(int(o["stream"]), int(o["comm"]), int(o["peer"]), int(o["didx"]),
                    int(prog.ops[r]["stream"]))].append((s, r))
    for lst in by_channel.values():
        lst.sort()
        for a in range(len(lst)):
            s1, r1 = lst[a]
            for b in range(a + 1, len(lst)):
                s2, r2 = lst[b]
                if r2 < r1 and accepts(prog, r2, s1):
                    bad.append(f"overtaking: send {s2} took recv {r2} ahead of earlier send {s1}")
    return bad


# ---------------------------------------------------------------------------
# exhaustive legal outcomes for tiny programs
# ---------------------------------------------------------------------------
def legal_outcomes(prog: Program, max_states: int = 2_000_000) -> Set[Tuple[FrozenSet, bool]]:
    """Every (match set, deadlocked) reachable under MPI semantics with eager
    sends: streams interleave freely; a send enters its (src, comm, dst)
    channel when posted and is delivered later in channel order; delivery
    matches the first posted receive of the domain that accepts it, a posted
    receive takes the first delivered-unmatched send that it accepts."""
    ops = prog.ops
    lo = [int(x) for x in prog.stream_op_lo]
    ns = prog.nstreams
    reqs = {}
    for j in range(len(ops)):
        if int(ops[j]["kind"]) in (WAIT, WAITALL):
            a = int(ops[j]["req_lo"])
            reqs[j] = [int(q) for q in prog.reqlist[a: a + int(ops[j]["req_n"])]]
        assert int(ops[j]["kind"]) not in (ALLREDUCE, AXPY)
    member = {j: comm_member(prog, int(ops[j]["comm"]), int(ops[j]["stream"]))
              for j in range(len(ops)) if int(ops[j]["comm"]) >= 0}

    def dom_of_send(s):
        return (int(ops[s]["comm"]), int(ops[s]["peer"]), int(ops[s]["didx"]))

    def dom_of_recv(r):
        return (int(ops[r]["comm"]),) + member[r]

    def chan_of(s):
        return (int(ops[s]["stream"]), int(ops[s]["comm"]), int(ops[s]["peer"]), int(ops[s]["didx"]))

    def ok(r, s):
        return (int(ops[r]["peer"]) in (ANY_SOURCE, member[s][0])) and \
               (int(ops[r]["sidx"]) in (ANY_INDEX, member[s][1])) and \
               (int(ops[r]["tag"]) in (ANY_TAG, int(ops[s]["tag"])))

    # state: (cursors, posted_recv_ops, chans, posted(dom->tuple), unexp(dom->tuple), matches)
    start = (tuple(lo[:-1]), frozenset(), (), (), (), frozenset())
    results = set()
    seen = set()
    stack = [start]
    while stack:
        st = stack.pop()
        if st in seen:
            continue
        seen.add(st)
        if len(seen) > max_states:
            raise RuntimeError("state space too large")
        cur, rposted, chans, posted, unexp, matches = st
        chans_d, posted_d, unexp_d = dict(chans), dict(posted), dict(unexp)
        matched = {x for pr in matches for x in pr}
        complete = lambda q: (int(ops[q]["kind"]) in SEND_KINDS and q < cur[int(ops[q]["stream"])]) or q in matched
        succ = []

        def pack_state(cur2, rposted2, chans2, posted2, unexp2, matches2):
            f = lambda d: tuple(sorted((k, v) for k, v in d.items() if v))
            return (tuple(cur2), frozenset(rposted2), f(chans2), f(posted2), f(unexp2), frozenset(matches2))

        def post_recv(r, posted2, unexp2, matches2):
            d = dom_of_recv(r)
            q = list(unexp2.get(d, ()))
            for i, s in enumerate(q):
                if ok(r, s):
                    del q[i]
                    unexp2[d] = tuple(q)
                    matches2.add((s, r))
                    return
            posted2[d] = posted2.get(d, ()) + (r,)

        for g in range(ns):
            j = cur[g]
            if j >= lo[g + 1]:
                continue
            k = int(ops[j]["kind"])
            cur2 = list(cur)
            chans2, posted2, unexp2, matches2 = dict(chans_d), dict(posted_d), dict(unexp_d), set(matches)
            rposted2 = set(rposted)
            if k in SEND_KINDS:
                c = chan_of(j)
                chans2[c] = chans2.get(c, ()) + (j,)
                cur2[g] += 1
            elif k == IRECV:
                post_recv(j, posted2, unexp2, matches2)
                cur2[g] += 1
            elif k == RECV:
                if j not in rposted:
                    post_recv(j, posted2, unexp2, matches2)
                    rposted2.add(j)
                elif j in matched:
                    cur2[g] += 1
                else:
                    continue
            elif k in (WAIT, WAITALL):
                if all(complete(q) for q in reqs[j]):
                    cur2[g] += 1
                else:
                    continue
            succ.append(pack_state(cur2, rposted2, chans2, posted2, unexp2, matches2))
        for c, q in chans_d.items():
            if not q:
                continue
            s = q[0]
            chans2, posted2, unexp2, matches2 = dict(chans_d), dict(posted_d), dict(unexp_d), set(matches)
            chans2[c] = q[1:]
            d = dom_of_send(s)
            pl = list(posted2.get(d, ()))
            for i, r in enumerate(pl):
                if ok(r, s):
                    del pl[i]
                    posted2[d] = tuple(pl)
                    matches2.add((s, r))
                    break
            else:
                unexp2[d] = unexp2.get(d, ()) + (s,)
            succ.append(pack_state(list(cur), rposted, chans2, posted2, unexp2, matches2))
        if not succ:
            dead = any(cur[g] < lo[g + 1] for g in range(ns))
            results.add((matches, dead))
        stack.extend(succ)
    return results


def match_set(match: np.ndarray, prog: Program) -> FrozenSet:
    kinds = prog.ops["kind"]
    return frozenset((s, int(match[s])) for s in range(len(match))
                     if kinds[s] in SEND_KINDS and match[s] >= 0)


# ---------------------------------------------------------------------------
# the outcome of a run whose matching may legally differ (live traffic)
# ---------------------------------------------------------------------------
def status_slot_of(prog: Program) -> Dict[int, int]:
    """Receive op -> the status slot a wait or waitall (or the receive itself)
    writes for it."""
    slot = {}
    kinds = prog.ops["kind"]
    for j, o in enumerate(prog.ops):
        k = int(kinds[j])
        if k == RECV and int(o["status"]) >= 0:
            slot[j] = int(o["status"])
        elif k in (WAIT, WAITALL) and int(o["status"]) >= 0:
            lo, n = int(o["req_lo"]), int(o["req_n"])
            for q in range(n):
                slot[int(prog.reqlist[lo + q])] = int(o["status"]) + q
    return slot


def infer_match_from_payloads(prog: Program, buffers, status) -> Tuple[np.ndarray, List[str]]:
    """The match map a run produced, read from what it delivered: each
    receive's status names (source, tag, bytes), and among the sends on that
    channel the one whose packed payload begins with the delivered bytes is
    its partner.  Needs payloads that tell sends apart (random bytes).
    Returns (match, problems): problems lists receives whose status or bytes
    no send explains, or a send claimed twice."""
    kinds = prog.ops["kind"]
    init = prog.fresh_buffers()
    types = prog.types
    match = np.full(len(prog.ops), -1, np.int64)
    problems = []
    by_channel = defaultdict(list)
    for s in np.nonzero(np.isin(kinds, SEND_KINDS))[0]:
        o = prog.ops[s]
        c = int(o["comm"])
        src, _ = comm_member(prog, c, int(o["stream"]))
        by_channel[(c, src, int(o["peer"]), int(o["tag"]))].append(int(s))
    slots = status_slot_of(prog)
    for r in np.nonzero(np.isin(kinds, RECV_KINDS))[0]:
        r = int(r)
        if r not in slots:
            problems.append(f"recv {r}: no status slot")
            continue
        st = status[slots[r]]
        o = prog.ops[r]
        c = int(o["comm"])
        dst, _ = comm_member(prog, c, int(o["stream"]))
        n = int(st["bytes"])
        got = np_pack(buffers[int(o["buf"])], int(o["off"]), types, int(o["type"]), int(o["count"]))[:n]
        cands = []
        for s in by_channel.get((c, int(st["source"]), dst, int(st["tag"])), []):
            so = prog.ops[s]
            sent = np_pack(init[int(so["buf"])], int(so["off"]), types, int(so["type"]), int(so["count"]))
            if len(sent) >= n and np.array_equal(sent[:n], got) and match[s] < 0:
                cands.append((s, len(sent)))
        if len(cands) != 1:
            problems.append(f"recv {r}: {len(cands)} sends explain status {tuple(st)}")
            continue
        s, sent_n = cands[0]
        cap = len(np_pack(init[int(o["buf"])], int(o["off"]), types, int(o["type"]), int(o["count"])))
        want_err = ERR_TRUNCATE if sent_n > cap else 0   # MPI truncation
        if n != min(sent_n, cap) or int(st["error"]) != want_err:
            problems.append(f"recv {r}: bytes {n} / error {int(st['error'])} do not fit send {s}")
        match[s], match[r] = r, s
    return match, problems
