"""Pins for the CPU oracle: each test checks it against something other than
itself (worked examples of the paper, closed forms, exhaustive enumeration of
legal MPI outcomes, exact integer arithmetic, independent numpy formulations).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from traffic import gen
from traffic.program import (ANY_SOURCE, ANY_TAG, ERR_TRUNCATE, IN_PLACE, MODE_FIXED, MODE_TREE,
                             T_BYTE, T_DOUBLE, T_FLOAT, T_INT32, T_INT64, ProgramBuilder)

from checks import (closed_form_matches, legal_outcomes, match_set, np_pack, np_unpack,
                    validity_violations)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_kv(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


# ---------------------------------------------------------------------------
# worked examples of the paper (§6)
# ---------------------------------------------------------------------------
def test_listing4_saxpy_gives_four():
    kv = _golden_kv("listing4.txt")
    p = gen.listing4(1 << 20, a=kv["a_val"], x_val=kv["x_val"], y_val=kv["y_val"])
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    y = o.buffers[p.meta["dy"]].view(np.float32)
    assert np.all(y == np.float32(kv["y_expected"]))
    # the received x is intact in rank 1's device buffer
    assert np.all(o.buffers[p.meta["dx"]].view(np.float32) == np.float32(kv["x_val"]))


def test_listing3_four_threads_deliver_100_bytes():
    p = gen.listing3(4, 100)
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    for s, d in zip(p.meta["src"], p.meta["dst"]):
        assert np.array_equal(o.buffers[d], p.buf_init[s])


# ---------------------------------------------------------------------------
# datatypes: hand-worked vector layouts and the 2-D slice formulation
# ---------------------------------------------------------------------------
def _golden_vectors():
    rows = []
    for line in open(os.path.join(GOLDEN, "vector_layout.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            lhs, rhs = line.split("|")
            vc, bl, st, cnt = (int(x) for x in lhs.split())
            rows.append((vc, bl, st, cnt, [int(x) for x in rhs.split()]))
    return rows


@pytest.mark.parametrize("row", _golden_vectors())
def test_vector_layout_worked_examples(row):
    vc, bl, st, cnt, expect = row
    b = ProgramBuilder(2)
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    src = b.buffer(np.arange(24, dtype=np.uint8))
    dst = b.buffer(64)
    t = b.vector(vc, bl, st, T_BYTE)
    b.send(g0, c, src, 0, cnt, t, 1, 0)
    b.recv(g1, c, dst, 0, len(expect), T_BYTE, 0, 0)
    p = b.build()
    o = oracle.run(p)
    assert o.error == 0
    assert list(o.buffers[dst][: len(expect)]) == expect
    assert np.all(o.buffers[dst][len(expect):] == 0)
    # the 2-D slice formulation agrees with the hand-worked bytes
    assert list(np_pack(np.arange(24, dtype=np.uint8), 0, p.types, t, cnt)) == expect


def test_vector_to_vector_unpack_matches_2d_slices():
    rng = np.random.default_rng(7)
    for trial in range(20):
        vc1, bl1 = int(rng.integers(1, 6)), int(rng.integers(1, 5))
        st1 = bl1 + int(rng.integers(0, 4))
        elem_t = [T_BYTE, T_INT32, T_FLOAT, T_INT64][trial % 4]
        esz = {T_BYTE: 1, T_INT32: 4, T_FLOAT: 4, T_INT64: 8}[elem_t]
        cnt1 = int(rng.integers(1, 4))
        nbytes = vc1 * bl1 * esz * cnt1
        # receive side: a different vector whose packed size is >= nbytes
        bl2 = int(rng.integers(1, 4))
        st2 = bl2 + int(rng.integers(0, 3))
        per2 = bl2 * esz
        vc2 = max(1, -(-nbytes // per2))
        b = ProgramBuilder(2)
        g0, g1 = b.stream(0), b.stream(1)
        c = b.comm([g0, g1])
        srcbytes = rng.integers(0, 256, 4096).astype(np.uint8)
        src = b.buffer(srcbytes)
        dst = b.buffer(rng.integers(0, 256, 4096).astype(np.uint8))
        t1 = b.vector(vc1, bl1, st1, elem_t)
        t2 = b.vector(vc2, bl2, st2, elem_t)
        b.send(g0, c, src, 8, cnt1, t1, 1, 3)
        b.recv(g1, c, dst, 16, 1, t2, 0, 3)
        p = b.build()
        o = oracle.run(p)
        assert o.error == 0
        expect = p.buf_init[dst].copy()
        np_unpack(expect, 16, p.types, t2, 1, np_pack(srcbytes, 8, p.types, t1, cnt1))
        assert np.array_equal(o.buffers[dst], expect), trial


def test_truncation_takes_capacity_and_reports_error():
    b = ProgramBuilder(2)
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    src = b.buffer(np.arange(1, 41, dtype=np.uint8))
    dst = b.buffer(np.full(64, 0xEE, np.uint8))
    st = b.status_slots(1)
    b.send(g0, c, src, 0, 10, T_INT32, 1, 5)
    b.recv(g1, c, dst, 4, 6, T_INT32, 0, 5, st)
    p = b.build()
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    d = o.buffers[dst]
    assert np.all(d[:4] == 0xEE) and np.all(d[28:] == 0xEE)     # canaries untouched
    assert np.array_equal(d[4:28], np.arange(1, 25, dtype=np.uint8))
    s = o.status[st]
    assert (s["source"], s["tag"], s["error"], s["bytes"]) == (0, 5, ERR_TRUNCATE, 24)


def test_zero_count_messages_match_in_order_and_move_nothing():
    """MPI: a message of count 0 matches like any other (by source, tag and
    order); it moves no bytes and its status carries the source, the tag and
    0 bytes.  A receive of capacity 0 that takes a longer message delivers
    nothing and reports MPI_ERR_TRUNCATE."""
    b = ProgramBuilder(2)
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    src = b.buffer(np.arange(1, 17, dtype=np.uint8))
    dst = b.buffer(np.full(16, 0xEE, np.uint8))
    st = b.status_slots(3)
    b.send(g0, c, src, 0, 0, T_FLOAT, 1, 7)                     # op 0: empty, tag 7
    b.send(g0, c, src, 0, 4, T_BYTE, 1, 7)                      # op 1: 4 bytes, tag 7
    b.send(g0, c, src, 4, 2, T_INT32, 1, 9)                     # op 2: 8 bytes, tag 9
    b.recv(g1, c, dst, 0, 4, T_BYTE, 0, 7, st)                  # op 3: the first tag-7 message
    b.recv(g1, c, dst, 0, 4, T_BYTE, ANY_SOURCE, ANY_TAG, st + 1)  # op 4: the next message
    b.recv(g1, c, dst, 8, 0, T_INT32, 0, 9, st + 2)             # op 5: capacity 0
    p = b.build()
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    assert [int(o.match[k]) for k in range(3)] == [3, 4, 5]
    got = [(int(s["source"]), int(s["tag"]), int(s["error"]), int(s["bytes"]))
           for s in o.status[st: st + 3]]
    assert got == [(0, 7, 0, 0), (0, 7, 0, 4), (0, 9, ERR_TRUNCATE, 0)]
    expect = np.full(16, 0xEE, np.uint8)
    expect[:4] = [1, 2, 3, 4]
    assert np.array_equal(o.buffers[dst], expect)


# ---------------------------------------------------------------------------
# matching: closed form, exhaustive enumeration, invariants
# ---------------------------------------------------------------------------
def _assert_closed_form(p, o):
    cf = closed_form_matches(p)
    got = {s: int(o.match[s]) for s in cf}
    assert got == cf
    nsend = sum(1 for j in range(len(p.ops)) if p.ops[j]["kind"] in (0, 2))
    assert len(cf) == nsend


def test_tiny_pairs_closed_form_and_payloads():
    p = gen.tiny_pairs(nmsg=300)
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    _assert_closed_form(p, o)
    # every receive lands at its message's offset: the arenas end up equal
    assert np.array_equal(o.buffers[p.meta["rbuf"]], p.buf_init[p.meta["sbuf"]])
    assert validity_violations(p, o.match, require_complete=True) == []
    # statuses: source 0, the message's tag, its full size
    counts, tags, order = p.meta["counts"], p.meta["tags"], p.meta["recv_order"]
    for i, m in enumerate(order):
        s = o.status[i]
        assert (s["source"], s["tag"], s["error"], s["bytes"]) == (0, tags[m], 0, 4 * counts[m])


def test_wildcard_free_random_programs_follow_closed_form():
    for seed in range(40):
        p = gen.random_small(seed, nranks=3, nmsg=6, p_any_src=0.0, p_any_tag=0.0)
        o = oracle.run(p)
        assert o.error == 0
        if not o.deadlock:
            _assert_closed_form(p, o)


@pytest.mark.parametrize("seed", range(60))
def test_outcome_is_among_all_legal_outcomes(seed):
    p = gen.random_small(seed, nranks=3, nmsg=5 if seed % 3 else 6)
    o = oracle.run(p)
    assert o.error == 0
    legal = legal_outcomes(p)
    assert (match_set(o.match, p), o.deadlock) in legal
    # the validity checker accepts every legal outcome of a finished run
    for ms, dead in legal:
        m = np.full(len(p.ops), -1, np.int64)
        for s, r in ms:
            m[s], m[r] = r, s
        assert validity_violations(p, m, require_complete=not dead) == []


def test_validity_checker_rejects_overtaking():
    # two sends on one channel, tag 0 then tag 0; receives take them crosswise
    b = ProgramBuilder(2)
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    s = b.buffer(16)
    r = b.buffer(16)
    b.isend(g0, c, s, 0, 1, T_INT32, 1, 0)
    b.isend(g0, c, s, 4, 1, T_INT32, 1, 0)
    b.irecv(g1, c, r, 0, 1, T_INT32, 0, ANY_TAG)
    b.irecv(g1, c, r, 4, 1, T_INT32, 0, 0)
    p = b.build()
    crossed = np.array([3, 2, 1, 0], np.int64)
    assert validity_violations(p, crossed, True)
    o = oracle.run(p)
    assert list(o.match) == [2, 3, 0, 1]


def test_any_source_takes_lowest_stream_first_in_round():
    # ranks 1 and 2 both send to rank 0 (tag 0) which posts ANY_SOURCE first
    b = ProgramBuilder(3)
    g = [b.stream(r) for r in range(3)]
    c = b.comm(g)
    s1, s2 = b.buffer(np.full(4, 1, np.uint8)), b.buffer(np.full(4, 2, np.uint8))
    r = b.buffer(8)
    b.irecv(g[0], c, r, 0, 4, T_BYTE, ANY_SOURCE, 0)
    b.irecv(g[0], c, r, 4, 4, T_BYTE, ANY_SOURCE, 0)
    b.send(g[2], c, s2, 0, 4, T_BYTE, 0, 0)
    b.send(g[1], c, s1, 0, 4, T_BYTE, 0, 0)
    p = b.build()
    o = oracle.run(p)
    # posts of round 1 in key order: rank0's two receives, rank1's send, rank2's send
    assert list(o.buffers[r]) == [1] * 4 + [2] * 4
    assert (match_set(o.match, p), False) in legal_outcomes(p)  # and MPI allows it


@pytest.mark.parametrize("seed", range(24))
def test_any_source_one_round_closed_form(seed):
    """Reading A1/A2 fixed for a whole family.  Every rank posts only
    nonblocking calls before its waitall, so everything is posted in round 1
    with key (1, stream id, program index); rank q posts M receives with
    (ANY_SOURCE, ANY_TAG) and the others send it M messages in all.  Sends from
    streams before q's wait as unexpected messages in key order and q's
    receives take them in that order; the later streams' sends find q's
    remaining receives in posting order.  Either way receive j takes the j-th
    send to q in (stream id, program index) order, wherever q's stream sits;
    stream ids are drawn independently of ranks, so rank order cannot stand in
    for it."""
    rng = np.random.default_rng(0x5EED + seed)
    R = int(rng.integers(3, 7))
    q = int(rng.integers(0, R))
    b = ProgramBuilder(R)
    gid = {}
    for r in rng.permutation(R):
        gid[int(r)] = b.stream(int(r))
    c = b.comm([gid[r] for r in range(R)])
    sends = []                  # (stream id, program index, rank, tag, payload)
    val = 1
    reqs = {r: [] for r in range(R)}
    for r in range(R):
        if r == q:
            continue
        for _ in range(int(rng.integers(0, 4))):
            n = int(rng.integers(1, 9))
            payload = np.arange(val, val + n, dtype=np.int32)
            val += n
            tag = int(rng.integers(0, 4))
            h = b.isend(gid[r], c, b.buffer(payload), 0, n, T_INT32, q, tag)
            reqs[r].append(h)
            sends.append((gid[r], h[1], r, tag, payload))
    M = len(sends)
    rbuf = b.buffer(np.full(8 * max(M, 1), -1, np.int32))
    for j in range(M):
        reqs[q].append(b.irecv(gid[q], c, rbuf, 32 * j, 8, T_INT32, ANY_SOURCE, ANY_TAG))
    st = b.status_slots(max(M, 1))
    for r in range(R):
        if reqs[r]:
            b.waitall(gid[r], reqs[r], st if r == q else -1)
    p = b.build()
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    order = sorted(sends, key=lambda x: (x[0], x[1]))
    got = o.buffers[rbuf].view(np.int32)
    for j, (g, k, r, tag, payload) in enumerate(order):
        recv_op = int(p.stream_op_lo[gid[q]]) + j
        assert int(o.match[int(p.stream_op_lo[g]) + k]) == recv_op
        n = len(payload)
        assert np.array_equal(got[8 * j: 8 * j + n], payload) and np.all(got[8 * j + n: 8 * j + 8] == -1)
        s_ = o.status[st + j]
        assert (int(s_["source"]), int(s_["tag"]), int(s_["error"]), int(s_["bytes"])) == (r, tag, 0, 4 * n)
    assert validity_violations(p, o.match, require_complete=True) == []


def test_round_model_hand_worked_wildcard_order():
    """Hand-worked under the round reading: rank 0 isends A then waits, then
    sends C; rank 1 sends B; rank 2 posts three ANY_SOURCE receives.
    Round 1 posts A (rank 0 then blocks: A completes at the end of round 1),
    B, and the three receives; in key order A and B are unexpected when R1 and
    R2 arrive, so R1<-A, R2<-B.  Round 2 posts C, which takes R3."""
    b = ProgramBuilder(3)
    g = [b.stream(r) for r in range(3)]
    c = b.comm(g)
    a = b.buffer(np.full(4, 0xA, np.uint8))
    bb = b.buffer(np.full(4, 0xB, np.uint8))
    cc = b.buffer(np.full(4, 0xC, np.uint8))
    r = b.buffer(12)
    h = b.isend(g[0], c, a, 0, 4, T_BYTE, 2, 0)
    b.wait(g[0], h)
    b.send(g[0], c, cc, 0, 4, T_BYTE, 2, 0)
    b.send(g[1], c, bb, 0, 4, T_BYTE, 2, 0)
    for k in range(3):
        b.irecv(g[2], c, r, 4 * k, 4, T_BYTE, ANY_SOURCE, 0)
    p = b.build()
    o = oracle.run(p)
    assert not o.deadlock
    assert list(o.buffers[r]) == [0xA] * 4 + [0xB] * 4 + [0xC] * 4
    assert list(o.post_round[:3]) == [1, 2, 2]
    assert (match_set(o.match, p), False) in legal_outcomes(p)  # and MPI allows it


def test_round_model_causal_order_beats_stream_order():
    """Hand-worked: rank 1 first receives from rank 2 (blocking) and only then
    sends P to rank 0; rank 2 sends Q to rank 0 and then T to rank 1; rank 0
    posts two ANY_SOURCE receives R1, R2 and waits for both.
    Round 1 posts, in key order (stream, then program order): R1, R2 (rank 0),
    rank 1's receive, Q and T (rank 2).  Q finds R1 posted and takes it; T
    completes rank 1's receive at the end of round 1.  Round 2 posts P, which
    takes R2.  So R1 <- Q (source 2) and R2 <- P (source 1), although rank 1's
    stream precedes rank 2's: the round (causal) order decides before the
    stream id.  MPI allows the other assignment too, so this pins the reading,
    not MPI alone: both assignments are among the enumerated legal outcomes."""
    b = ProgramBuilder(3)
    g = [b.stream(r) for r in range(3)]
    c = b.comm(g)
    pbuf = b.buffer(np.full(4, 0x11, np.uint8))
    qbuf = b.buffer(np.full(4, 0x22, np.uint8))
    tbuf = b.buffer(np.full(4, 0x33, np.uint8))
    rbuf = b.buffer(8)
    x = b.buffer(4)
    st = b.status_slots(2)
    h1 = b.irecv(g[0], c, rbuf, 0, 4, T_BYTE, ANY_SOURCE, 0)
    h2 = b.irecv(g[0], c, rbuf, 4, 4, T_BYTE, ANY_SOURCE, 0)
    b.waitall(g[0], [h1, h2], st)
    b.recv(g[1], c, x, 0, 4, T_BYTE, 2, 5)
    b.send(g[1], c, pbuf, 0, 4, T_BYTE, 0, 0)
    b.send(g[2], c, qbuf, 0, 4, T_BYTE, 0, 0)
    b.send(g[2], c, tbuf, 0, 4, T_BYTE, 1, 5)
    p = b.build()
    o = oracle.run(p)
    assert not o.deadlock and o.error == 0
    assert list(o.buffers[rbuf]) == [0x22] * 4 + [0x11] * 4
    assert [int(v) for v in o.status["source"][st: st + 2]] == [2, 1]
    legal = legal_outcomes(p)
    outcomes = {ms for ms, dead in legal if not dead}
    assert match_set(o.match, p) in outcomes and len(outcomes) == 2


def test_round_model_wildcard_patterns_in_key_order():
    """Hand-worked, one round: rank 0 posts R1 (source 1, tag 7), R2 (ANY_SOURCE,
    ANY_TAG), R3 (ANY_SOURCE, tag 7), R4 (source 2, tag 3), then waits; rank 1
    sends A and B (tag 7); rank 2 sends C (tag 3) and D (tag 7).  In key order
    the receives are posted first; A takes the first receive accepting
    (1, 7), R1; B takes R2 (R1 is gone, R2 accepts anything); C (2, 3) skips
    R3 (tag 7) and takes R4; D takes R3."""
    b = ProgramBuilder(3)
    g = [b.stream(r) for r in range(3)]
    c = b.comm(g)
    src = {k: b.buffer(np.full(2, v, np.uint8)) for k, v in zip("ABCD", (0xA, 0xB, 0xC, 0xD))}
    rbuf = b.buffer(8)
    st = b.status_slots(4)
    pats = [(1, 7), (ANY_SOURCE, ANY_TAG), (ANY_SOURCE, 7), (2, 3)]
    hs = [b.irecv(g[0], c, rbuf, 2 * k, 2, T_BYTE, s_, t_) for k, (s_, t_) in enumerate(pats)]
    b.waitall(g[0], hs, st)
    b.send(g[1], c, src["A"], 0, 2, T_BYTE, 0, 7)
    b.send(g[1], c, src["B"], 0, 2, T_BYTE, 0, 7)
    b.send(g[2], c, src["C"], 0, 2, T_BYTE, 0, 3)
    b.send(g[2], c, src["D"], 0, 2, T_BYTE, 0, 7)
    p = b.build()
    o = oracle.run(p)
    assert not o.deadlock and o.error == 0
    assert list(o.buffers[rbuf]) == [0xA] * 2 + [0xB] * 2 + [0xD] * 2 + [0xC] * 2
    s = o.status[st: st + 4]
    assert [int(v) for v in s["source"]] == [1, 1, 2, 2]
    assert [int(v) for v in s["tag"]] == [7, 7, 7, 3]
    legal = legal_outcomes(p)
    assert (match_set(o.match, p), False) in legal


def test_send_request_status_is_the_empty_status():
    """A wait on a send request writes MPI's empty status (fixture with its
    citation), as does every send entry of a waitall; a receive entry of the
    same waitall carries the message's source, tag and bytes."""
    empty = _golden_kv("empty_status.txt")
    b = ProgramBuilder(2)
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    sbuf = b.buffer(np.arange(32, dtype=np.uint8))
    rbuf = b.buffer(32)
    st = b.status_slots(3)
    h = b.isend(g0, c, sbuf, 0, 4, T_INT32, 1, 9)
    b.wait(g0, h, st)
    h2 = b.isend(g1, c, sbuf, 16, 2, T_INT32, 0, 4)
    h3 = b.irecv(g1, c, rbuf, 0, 4, T_INT32, 0, 9)
    b.waitall(g1, [h2, h3], st + 1)
    b.recv(g0, c, rbuf, 16, 2, T_INT32, 1, 4)
    p = b.build()
    o = oracle.run(p)
    assert not o.deadlock and o.error == 0
    for k in (0, 1):
        s = o.status[st + k]
        assert (int(s["source"]), int(s["tag"]), int(s["error"]), int(s["bytes"])) == \
            (empty["source"], empty["tag"], empty["error"], empty["bytes"])
    r = o.status[st + 2]
    assert (int(r["source"]), int(r["tag"]), int(r["error"]), int(r["bytes"])) == (0, 9, 0, 16)


def test_deadlock_detected_on_cyclic_blocking_receives():
    b = ProgramBuilder(2)
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    x = b.buffer(16)
    j0 = b.recv(g0, c, x, 0, 1, T_INT32, 1, 0)
    b.send(g0, c, x, 4, 1, T_INT32, 1, 0)
    j1 = b.recv(g1, c, x, 8, 1, T_INT32, 0, 0)
    b.send(g1, c, x, 12, 1, T_INT32, 0, 0)
    p = b.build()
    o = oracle.run(p)
    assert o.deadlock
    assert list(o.stuck_op) == [0, 2]


def test_eager_send_snapshot_taken_at_post():
    # the sender overwrites its buffer (axpy) after a blocking send; the
    # receiver posts late and must see the bytes of the send's moment
    b = ProgramBuilder(2)
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    xs = b.buffer(np.ones(8, np.float32))
    ys = b.buffer(np.full(8, 3.0, np.float32))
    r = b.buffer(32)
    scratch = b.buffer(64)
    b.send(g0, c, ys, 0, 8, T_FLOAT, 1, 0)
    b.axpy(g0, 2.0, xs, 0, ys, 0, 8)
    b.recv(g1, c, scratch, 0, 1, T_INT32, 0, 9)   # unmatched first: blocks rank 1
    b.recv(g1, c, r, 0, 8, T_FLOAT, 0, 0)
    p = b.build()
    o = oracle.run(p)
    assert o.deadlock  # rank 1 is stuck on tag 9, by construction
    assert np.all(o.buffers[ys].view(np.float32) == 5.0)


def test_ring_exchange_matches_numpy_restatement():
    """An independent numpy formulation of the ring workload: closed-form
    neighbours, axpy with alpha=0.5 (exact product, one rounding in the add),
    vector layouts as 2-D slices."""
    steps, n = 6, 1 << 12
    p = gen.ring_exchange(nranks=5, n=n, steps=steps, min_bytes=256, max_bytes=1 << 15)
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    _assert_closed_form(p, o)
    bufs = p.fresh_buffers()
    S, RL, RR = p.meta["S"], p.meta["RL"], p.meta["RR"]
    R = 5
    ops = p.ops
    # walk the per-step structure: [axpy, isend, isend, irecv, irecv, waitall]
    per = 6
    for step in range(steps):
        for r in range(R):
            x = bufs[RL[r]].view(np.float32)[:n]
            y = bufs[S[r]].view(np.float32)
            y[:n] = (np.float32(0.5) * x + y[:n]).astype(np.float32)
        msgs = []
        for r in range(R):
            base = int(p.stream_op_lo[r]) + step * per
            for d in range(2):
                so = ops[base + 1 + d]
                msgs.append((r, d, np_pack(bufs[S[r]], 0, p.types, int(so["type"]), int(so["count"]))))
        for r, d, data in msgs:
            dest = (r + 1) % R if d == 0 else (r - 1) % R
            base = int(p.stream_op_lo[dest]) + step * per
            ro = ops[base + 3 + d]
            tgt = RL[dest] if d == 0 else RR[dest]
            np_unpack(bufs[tgt], 0, p.types, int(ro["type"]), int(ro["count"]), data)
    for k in range(len(bufs)):
        assert np.array_equal(o.buffers[k], bufs[k]), k


# ---------------------------------------------------------------------------
# allreduce
# ---------------------------------------------------------------------------
def _instances(p, o):
    for inst in p.meta["instances"]:
        xs = [p.buf_init[inst["recv"][r]] if inst["send"][r] == IN_PLACE else p.buf_init[inst["send"][r]]
              for r in range(p.nranks)]
        outs = [o.buffers[b] for b in inst["recv"]]
        yield inst, xs, outs


def test_allreduce_integers_equal_exact_sums():
    p = gen.allreduce_suite(nranks=5, sizes=(1, 33), dtypes=(T_INT64, T_INT32, T_BYTE))
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    for inst, xs, outs in _instances(p, o):
        dt = inst["dtype"]
        npt, bits = {T_INT64: (np.int64, 64), T_INT32: (np.int32, 32), T_BYTE: (np.uint8, 8)}[dt]
        vals = [x.view(npt).astype(object) for x in xs]
        for i in range(inst["n"]):
            exact = sum(int(v[i]) for v in vals) % (1 << bits)
            for out in outs:
                got = int(out.view(npt)[i]) % (1 << bits)
                assert got == exact


def test_allreduce_int64_wraps_near_2_63():
    b = ProgramBuilder(3)
    g = [b.stream(r) for r in range(3)]
    c = b.comm(g)
    big = np.array([(1 << 63) - 5, -(1 << 63) + 2, 7], np.int64)
    sb = [b.buffer(np.array([big[r]], np.int64)) for r in range(3)]
    rb = [b.buffer(8) for r in range(3)]
    for r in range(3):
        b.allreduce(g[r], c, sb[r], 0, rb[r], 0, 1, T_INT64)
    p = b.build()
    o = oracle.run(p)
    exact = (int(big[0]) + int(big[1]) + int(big[2])) % (1 << 64)
    for r in range(3):
        assert int(o.buffers[rb[r]].view(np.uint64)[0]) == exact


def test_allreduce_fp32_fixed_is_left_fold():
    p = gen.allreduce_suite(nranks=16, sizes=(1000,), dtypes=(T_FLOAT,), modes=(MODE_FIXED,))
    o = oracle.run(p)
    for inst, xs, outs in _instances(p, o):
        fl = [x.view(np.float32) for x in xs]
        acc = fl[0].copy()
        for k in range(1, len(fl)):
            acc = np.add(acc, fl[k], dtype=np.float32)
        for out in outs:
            assert np.array_equal(out.view(np.float32), acc)
        # and the fold is within the sequential-summation bound of the exact sum
        gamma = (len(fl) - 1) * 2.0 ** -24 / (1 - (len(fl) - 1) * 2.0 ** -24)
        for i in range(0, 1000, 37):
            exact = math.fsum(float(f[i]) for f in fl)
            mag = sum(abs(float(f[i])) for f in fl)
            assert abs(float(acc[i]) - exact) <= gamma * mag + 1e-45


def test_allreduce_fp64_fixed_is_left_fold():
    """fp64 SUM in fixed order: ((x0 + x1) + x2) + ... in rank order, one
    rounding per addition, within the sequential-summation bound of the exact
    sum (Higham, Accuracy and Stability of Numerical Algorithms, §4.2)."""
    R, n = 16, 777
    p = gen.allreduce_suite(nranks=R, sizes=(n,), dtypes=(T_DOUBLE,), modes=(MODE_FIXED,))
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    for inst, xs, outs in _instances(p, o):
        fl = [x.view(np.float64) for x in xs]
        acc = fl[0].copy()
        for k in range(1, R):
            acc = acc + fl[k]
        for out in outs:
            assert np.array_equal(out.view(np.float64), acc)
        u = 2.0 ** -53
        gamma = (R - 1) * u / (1 - (R - 1) * u)
        for i in range(0, n, 7):
            exact = sum((Fraction(float(f[i])) for f in fl), Fraction(0))
            mag = sum(abs(float(f[i])) for f in fl)
            assert abs(Fraction(float(acc[i])) - exact) <= Fraction(gamma * mag)


def test_allreduce_fp32_tree_mode_and_reference_sum():
    p = gen.allreduce_suite(nranks=16, sizes=(512,), dtypes=(T_FLOAT,), modes=(MODE_TREE,),
                            in_place=True)
    o = oracle.run(p)
    for inst, xs, outs in _instances(p, o):
        fl = [x.view(np.float32) for x in xs]
        s64, a64 = oracle.sum_f32_ref(fl)
        for i in range(512):
            exact = Fraction(0)
            for f in fl:
                exact += Fraction(float(f[i]))
            # a double sum of 16 floats (24-bit mantissas within a few octaves) is exact
            assert abs(Fraction(s64[i]) - exact) <= Fraction(abs(a64[i])) * Fraction(16, 2 ** 53)
            assert a64[i] == math.fsum(abs(float(f[i])) for f in fl)
            assert float(outs[0].view(np.float32)[i]) == float(np.float32(float(exact)))


def test_axpy_single_rounding():
    # alpha = 0.5: the product is exact in fp32, so fma(a,x,y) == fl(fl(a*x) + y)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(4096).astype(np.float32)
    y = rng.standard_normal(4096).astype(np.float32)
    b = ProgramBuilder(1)
    g = b.stream(0)
    xb, yb = b.buffer(x), b.buffer(y)
    b.axpy(g, 0.5, xb, 0, yb, 0, 4096)
    p = b.build()
    o = oracle.run(p)
    assert np.array_equal(o.buffers[yb].view(np.float32), np.float32(0.5) * x + y)
    # a general alpha: compare with an exactly rounded rational computation
    b = ProgramBuilder(1)
    g = b.stream(0)
    xb, yb = b.buffer(x[:256]), b.buffer(y[:256])
    b.axpy(g, 0.3, xb, 0, yb, 0, 256)
    p = b.build()
    o = oracle.run(p)
    a = Fraction(float(np.float32(0.3)))
    got = o.buffers[yb].view(np.float32)
    for i in range(256):
        exact = a * Fraction(float(x[i])) + Fraction(float(y[i]))
        cand = np.float32(float(exact))          # nearest double, then nearest float
        lo_, hi_ = np.nextafter(cand, np.float32(-np.inf)), np.nextafter(cand, np.float32(np.inf))
        best = min((lo_, cand, hi_), key=lambda v: abs(Fraction(float(v)) - exact))
        assert got[i] == best


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by the pins above
# ---------------------------------------------------------------------------
MUTANTS = [
    # LIFO instead of FIFO scan of the unexpected queue
    ("for (auto it = lst.begin(); it != lst.end(); ++it) {\n      const Op& so",
     "for (auto it = lst.end(); it != lst.begin();) { --it;\n      const Op& so"),
    # tag test ignores ANY_TAG
    ("bool tag_ok = recv.tag == kAnyTag || recv.tag == tag;", "bool tag_ok = recv.tag == tag;"),
    # dropped last allreduce term
    ("for (size_t k = 1; k < R; ++k) acc += load<uint64_t>(in[k], i);",
     "for (size_t k = 1; k + 1 < R; ++k) acc += load<uint64_t>(in[k], i);"),
    # vector stride and blocklen swapped in the address formula
    ("return i * L.extent + (b * L.stride + j) * L.elem + within;",
     "return i * L.extent + (b * L.blocklen + j) * L.elem + within;"),
    # completions visible in the same round
    ("return r.done_round[j] >= 0 && r.done_round[j] < round;",
     "return r.done_round[j] >= 0 && r.done_round[j] <= round;"),
    # truncation reported on the wrong side
    ("st.error = sent > cap ? kErrTruncate : 0;", "st.error = sent < cap ? kErrTruncate : 0;"),
    # fp32 fixed-order fold over the ranks after the first in reverse order
    ("for (size_t k = 1; k < R; ++k) acc = acc + load<float>(in[k], i);",
     "for (size_t k = R - 1; k >= 1; --k) acc = acc + load<float>(in[k], i);"),
    # fp64 fixed-order fold drops the last rank's term
    ("for (size_t k = 1; k < R; ++k) acc = acc + load<double>(in[k], i);",
     "for (size_t k = 1; k + 1 < R; ++k) acc = acc + load<double>(in[k], i);"),
    # tree-mode reference sum drops rank 0's term
    ("for (size_t k = 0; k < R; ++k) acc += (double)load<float>(in[k], i);",
     "for (size_t k = 1; k < R; ++k) acc += (double)load<float>(in[k], i);"),
    # axpy rounded twice (product, then sum) instead of once
    ("y = std::fma(o.alpha, x, y);", "y = o.alpha * x + y;"),
    # a send request's status carries rank 0 instead of MPI_ANY_SOURCE
    ("st.source = kAnySource;  // empty status for send requests",
     "st.source = 0;  // empty status for send requests"),
]


@pytest.mark.parametrize("k", range(len(MUTANTS)))
def test_planted_mistake_is_caught(k, tmp_path, monkeypatch):
    import importlib
    import shutil
    src = open(os.path.join(os.path.dirname(oracle.__file__), "mpx_oracle.cpp")).read()
    old, new = MUTANTS[k]
    assert old in src
    d = tmp_path / "oracle"
    d.mkdir()
    (d / "mpx_oracle.cpp").write_text(src.replace(old, new, 1))
    shutil.copy(oracle.__file__, d / "__init__.py")
    import sys
    monkeypatch.syspath_prepend(str(tmp_path))
    saved = sys.modules.pop("oracle")
    try:
        mutant = importlib.import_module("oracle")
        assert mutant.__file__.startswith(str(tmp_path))
        monkeypatch.setitem(globals(), "oracle", mutant)
        checks = [test_listing4_saxpy_gives_four, test_tiny_pairs_closed_form_and_payloads,
                  test_allreduce_integers_equal_exact_sums, test_vector_to_vector_unpack_matches_2d_slices,
                  test_truncation_takes_capacity_and_reports_error,
                  test_validity_checker_rejects_overtaking, test_ring_exchange_matches_numpy_restatement,
                  test_round_model_hand_worked_wildcard_order, test_any_source_takes_lowest_stream_first_in_round,
                  test_zero_count_messages_match_in_order_and_move_nothing,
                  lambda: [test_any_source_one_round_closed_form(s) for s in range(24)],
                  test_allreduce_fp32_fixed_is_left_fold, test_allreduce_fp32_tree_mode_and_reference_sum,
                  test_allreduce_fp64_fixed_is_left_fold,
                  test_axpy_single_rounding, test_send_request_status_is_the_empty_status,
                  lambda: [test_outcome_is_among_all_legal_outcomes(s) for s in range(60)]]
        caught = False
        for fn in checks:
            try:
                fn()
            except AssertionError:
                caught = True
                break
        assert caught, f"mutant {k} survived"
    finally:
        sys.modules["oracle"] = saved


@pytest.mark.parametrize("k", range(12))
def test_laminar_batching_programs_complete_without_truncation(k):
    """The batching generator's laminar option (ANY_SOURCE receives are also
    ANY_TAG; receives posted most specific first; capacities the largest
    admissible message) yields programs every receive of which completes
    untruncated.  Checked here through the oracle at high wildcard rates."""
    from traffic import gen
    p = gen.batching(nranks=4, streams_per_rank=2, nmsg=60, max_bytes=256, ntags=3,
                     p_any_tag=0.3, p_any_source=0.3, laminar=True, seed=gen.SEED_BASE + 1000 + k)
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    assert np.all(o.status["error"] == 0)
