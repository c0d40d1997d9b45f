"""Pins of the oracle's multiplex stream communicator (§3.5).

Each check reaches the oracle's answer from something other than its code:
the brute-force enumerator of MPI-legal executions (tests/checks.py), the
wildcard-free closed form over (rank, local index) members, numpy
restatements of the payload movement, and a hand-worked example.  The
planted-mistake test at the end breaks the oracle's multiplex rules one at
a time and requires one of these checks to fail.
"""
from __future__ import annotations

import importlib
import os
import shutil
import sys

import numpy as np
import pytest

import oracle
from tests.checks import closed_form_matches, legal_outcomes, match_set, np_pack, validity_violations
from traffic import gen
from traffic.program import ANY_INDEX, ANY_SOURCE, ANY_TAG, T_INT32, ProgramBuilder


def _legal(seed):
    counts = (2, 3) if seed % 2 else (3, 1)
    p = gen.multiplex_small(gen.SEED_BASE + 700 + seed, nranks=2, counts=counts,
                            nmsg=5 if seed % 3 else 6)
    o = oracle.run(p)
    assert o.error == 0
    legal = legal_outcomes(p)
    assert (match_set(o.match, p), o.deadlock) in legal
    if not o.deadlock:
        assert validity_violations(p, o.match, require_complete=True) == []


@pytest.mark.parametrize("seed", range(40))
def test_multiplex_outcome_is_among_all_legal_outcomes(seed):
    _legal(seed)


def _closed_form(seed):
    """Without wildcards the k-th send from member a to member b with tag t
    matches the k-th receive b posts for (a, t); the receive's bytes are the
    send's packed bytes and its status names a's rank and index."""
    p = gen.multiplex_small(gen.SEED_BASE + 800 + seed, nranks=3, counts=(2, 1, 3), nmsg=12,
                            p_any_src=0.0, p_any_idx=0.0, p_any_tag=0.0, p_blocking=0.0, p_wait=0.0)
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    want = closed_form_matches(p)
    for s, r in want.items():
        assert o.match[s] == r
    assert (o.match >= 0).sum() == 2 * len(want)
    init = p.fresh_buffers()
    for s, r in want.items():
        so, ro = p.ops[s], p.ops[r]
        data = np_pack(init[int(so["buf"])], int(so["off"]), p.types, int(so["type"]), int(so["count"]))
        got = o.buffers[int(ro["buf"])][int(ro["off"]): int(ro["off"]) + len(data)]
        assert np.array_equal(got, data)


@pytest.mark.parametrize("seed", range(8))
def test_multiplex_wildcard_free_follows_closed_form(seed):
    _closed_form(seed)


def _n_to_one():
    """Every sender's messages reach the poller in order (tags 0, 1, ...),
    each exactly once, with its rank and index in the status and its bytes."""
    p = gen.n_to_one(nranks=3, threads=3, msgs=5, max_bytes=512)
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    st = o.status
    seen = {}
    for k in range(len(st)):
        key = (int(st["source"][k]), int(st["source_index"][k]))
        seen.setdefault(key, []).append(int(st["tag"][k]))
    senders = [(r, i) for r in range(3) for i in range(3) if (r, i) != (0, 0)]
    assert sorted(seen) == senders
    for key in senders:
        assert seen[key] == list(range(5)), (key, seen[key])
    # payloads: the poller's k-th receive holds the matched send's bytes
    init = p.fresh_buffers()
    rb = o.buffers[int(p.ops[int(np.nonzero(p.ops["kind"] == 3)[0][0])]["buf"])]
    for j in np.nonzero(p.ops["kind"] == 3)[0]:
        s = int(o.match[j])
        so, ro = p.ops[s], p.ops[int(j)]
        data = init[int(so["buf"])][int(so["off"]): int(so["off"]) + 4 * int(so["count"])]
        assert np.array_equal(rb[int(ro["off"]): int(ro["off"]) + len(data)], data)


def test_n_to_one_delivers_each_message_once_in_sender_order():
    _n_to_one()


def test_single_stream_comm_equals_multiplex_with_one_stream_per_rank():
    """A multiplex comm where every rank attaches one stream behaves like the
    plain stream comm over the same streams (every index is 0)."""
    for seed in range(6):
        p = gen.random_small(seed, nranks=3, nmsg=6)
        q = gen.random_small(seed, nranks=3, nmsg=6)
        q.comm_mux = [[[int(g)] for g in q.comm_stream[0]]]
        a, b = oracle.run(p), oracle.run(q)
        assert a.error == 0 and b.error == 0 and a.deadlock == b.deadlock
        assert np.array_equal(a.match, b.match)
        assert np.array_equal(a.status, b.status)
        for x, y in zip(a.buffers, b.buffers):
            assert np.array_equal(x, y)


def _hand_worked():
    """Rank 1 attaches streams 0 and 1, both send tag 0 to rank 0's stream 0
    (stream 0's send is posted first: lower stream id in the same round).
    Rank 0 posts (1, index 1, tag 0) and then (1, ANY_INDEX, tag 0), both
    nonblocking.  The first receive skips stream 0's earlier message: it
    matches index 1 only; the second takes stream 0's.  A third receive with
    (ANY_SOURCE, index 0) posted on rank 0's stream 1 matches nothing: no
    message targets that stream."""
    b = ProgramBuilder(2)
    g00, g01 = b.stream(0), b.stream(0)
    g10, g11 = b.stream(1), b.stream(1)
    c = b.comm_multiple([[g00, g01], [g10, g11]])
    sb0 = b.buffer(np.array([10, 11], np.int32))
    sb1 = b.buffer(np.array([20, 21], np.int32))
    rb = b.buffer(16)
    s0 = b.stream_send(g10, c, sb0, 0, 2, T_INT32, 0, 0, 0)
    s1 = b.stream_send(g11, c, sb1, 0, 2, T_INT32, 0, 0, 0)
    r1 = b.stream_recv(g00, c, rb, 0, 2, T_INT32, 1, 1, 0)
    r2 = b.stream_recv(g00, c, rb, 8, 2, T_INT32, 1, ANY_INDEX, 0)
    b.waitall(g10, [s0])
    b.waitall(g11, [s1])
    b.waitall(g00, [r1, r2], b.status_slots(2))
    b.stream_recv(g01, c, rb, 0, 2, T_INT32, ANY_SOURCE, 0, ANY_TAG, blocking=True)
    p = b.build()
    o = oracle.run(p)
    assert o.error == 0
    assert o.deadlock  # the lone receive on rank 0's stream 1 never completes
    assert o.buffers[rb][:16].view(np.int32).tolist() == [20, 21, 10, 11]
    assert [(int(x["source"]), int(x["source_index"]), int(x["bytes"])) for x in o.status] == \
        [(1, 1, 8), (1, 0, 8)]


def test_any_index_and_exact_index_hand_worked():
    _hand_worked()


MUX_MUTANTS = [
    # the source index pattern ignored
    ("bool idx_ok = recv.sidx == kAnyIndex || recv.sidx == src_index;", "bool idx_ok = true;"),
    # ANY_INDEX not honoured
    ("bool idx_ok = recv.sidx == kAnyIndex || recv.sidx == src_index;",
     "bool idx_ok = recv.sidx == src_index;"),
    # sends matched in the destination rank's domain regardless of its stream
    ("const Domain d{so.comm, so.peer, so.didx};", "const Domain d{so.comm, so.peer, 0};"),
    # status reports the receiver's own index
    ("st.source_index = op_index[(size_t)s];", "st.source_index = op_index[(size_t)q];"),
]


@pytest.mark.parametrize("k", range(len(MUX_MUTANTS)))
def test_planted_multiplex_mistake_is_caught(k, tmp_path, monkeypatch):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "mpx_oracle.cpp")).read()
    old, new = MUX_MUTANTS[k]
    assert old in src
    d = tmp_path / "oracle"
    d.mkdir()
    (d / "mpx_oracle.cpp").write_text(src.replace(old, new, 1))
    shutil.copy(oracle.__file__, d / "__init__.py")
    monkeypatch.syspath_prepend(str(tmp_path))
    saved = sys.modules.pop("oracle")
    try:
        mutant = importlib.import_module("oracle")
        assert mutant.__file__.startswith(str(tmp_path))
        monkeypatch.setitem(globals(), "oracle", mutant)
        checks = [_hand_worked, _n_to_one, lambda: [_closed_form(s) for s in range(4)],
                  lambda: [_legal(s) for s in range(20)]]
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


def test_multiplex_truncation_and_zero_count_statuses():
    """A receive shorter than the message takes its capacity and reports
    TRUNCATE; a zero-count message matches and delivers nothing; both
    statuses name the sender's rank and local index."""
    from traffic.program import ERR_TRUNCATE
    b = ProgramBuilder(2)
    g00 = b.stream(0)
    g10, g11 = b.stream(1), b.stream(1)
    c = b.comm_multiple([[g00], [g10, g11]])
    sb = b.buffer(np.arange(8, dtype=np.int32))
    rb = b.buffer(np.full(8, -1, np.int32))
    s1 = b.stream_send(g11, c, sb, 0, 8, T_INT32, 0, 0, 5)
    s0 = b.stream_send(g10, c, sb, 0, 0, T_INT32, 0, 0, 6)
    r1 = b.stream_recv(g00, c, rb, 0, 3, T_INT32, 1, 1, 5)
    r0 = b.stream_recv(g00, c, rb, 16, 4, T_INT32, ANY_SOURCE, ANY_INDEX, 6)
    b.waitall(g11, [s1])
    b.waitall(g10, [s0])
    b.waitall(g00, [r1, r0], b.status_slots(2))
    o = oracle.run(b.build())
    assert o.error == 0 and not o.deadlock
    assert o.buffers[rb].view(np.int32).tolist() == [0, 1, 2, -1, -1, -1, -1, -1]
    st = [(int(x["source"]), int(x["source_index"]), int(x["tag"]), int(x["error"]), int(x["bytes"]))
          for x in o.status]
    assert st == [(1, 1, 5, ERR_TRUNCATE, 12), (1, 0, 6, 0, 0)]


def test_multiplex_sender_order_is_kept_per_member_pair():
    """Non-overtaking per (sender member, receiver member): two messages from
    rank 1's stream 1 with one tag reach rank 0's stream 1 in send order even
    when the receives are (ANY_SOURCE, ANY_INDEX) and a message from another
    member arrives between them."""
    b = ProgramBuilder(2)
    g00, g01 = b.stream(0), b.stream(0)
    g10, g11 = b.stream(1), b.stream(1)
    c = b.comm_multiple([[g00, g01], [g10, g11]])
    bufs = [b.buffer(np.full(2, v, np.int32)) for v in (1, 2, 3)]
    rb = b.buffer(24)
    h1 = b.stream_send(g11, c, bufs[0], 0, 2, T_INT32, 0, 1, 0)
    h2 = b.stream_send(g10, c, bufs[1], 0, 2, T_INT32, 0, 1, 0)
    h3 = b.stream_send(g11, c, bufs[2], 0, 2, T_INT32, 0, 1, 0)
    rs = [b.stream_recv(g01, c, rb, 8 * k, 2, T_INT32, ANY_SOURCE, ANY_INDEX, 0) for k in range(3)]
    b.waitall(g11, [h1, h3])
    b.waitall(g10, [h2])
    b.waitall(g01, rs, b.status_slots(3))
    p = b.build()
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    got = o.buffers[rb].view(np.int32)[::2].tolist()
    assert got.index(1) < got.index(3)
    assert validity_violations(p, o.match, require_complete=True) == []
    legal = legal_outcomes(p)
    assert (match_set(o.match, p), False) in legal
