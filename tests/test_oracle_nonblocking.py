"""Pins of the oracle's nonblocking collectives (MPI_Iallreduce, MPI_Ibcast,
MPI_Ireduce, MPI_Iallgather in enqueue form, §3.4): the call lets its stream
go on at once and a later wait completes it.  Facts from MPI restated here:
a program that deadlocks with blocking collectives completes with
nonblocking ones; the results are those of the blocking definitions (exact
sums, copies, rank-ordered blocks); blocking and nonblocking calls share the
instance order but never match each other.  The planted mistakes at the end
must each fail one of these checks."""
import importlib
import os
import shutil
import sys

import numpy as np
import pytest

import oracle
from traffic.program import IN_PLACE, MODE_FIXED, T_INT32, T_INT64, ProgramBuilder


def _world(R):
    b = ProgramBuilder(R)
    gs = [b.stream(r) for r in range(R)]
    return b, gs, b.comm(gs)


def _crossing(nonblocking):
    """Rank 0: allreduce, then send to rank 1.  Rank 1: receive from rank 0,
    then allreduce.  Blocking allreduces wait for each other across the
    send/receive pair (a deadlock); nonblocking ones let both streams reach
    the pair, and each rank waits for its allreduce at the end."""
    b, gs, c = _world(2)
    x = [b.buffer(np.array([3 + r, 10 * r], np.int64)) for r in range(2)]
    y = [b.buffer(16) for _ in range(2)]
    msg, got = b.buffer(np.arange(4, dtype=np.int32)), b.buffer(16)
    if nonblocking:
        h0 = b.iallreduce(gs[0], c, x[0], 0, y[0], 0, 2, T_INT64)
        b.send(gs[0], c, msg, 0, 4, T_INT32, 1, 9)
        b.wait(gs[0], h0)
        b.recv(gs[1], c, got, 0, 4, T_INT32, 0, 9)
        h1 = b.iallreduce(gs[1], c, x[1], 0, y[1], 0, 2, T_INT64)
        b.wait(gs[1], h1)
    else:
        b.allreduce(gs[0], c, x[0], 0, y[0], 0, 2, T_INT64)
        b.send(gs[0], c, msg, 0, 4, T_INT32, 1, 9)
        b.recv(gs[1], c, got, 0, 4, T_INT32, 0, 9)
        b.allreduce(gs[1], c, x[1], 0, y[1], 0, 2, T_INT64)
    return b.build(), y, got


def _check_crossing():
    p, _, _ = _crossing(False)
    assert oracle.run(p).deadlock
    p, y, got = _crossing(True)
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    for r in range(2):
        assert o.buffers[y[r]].view(np.int64).tolist() == [3 + 4, 0 + 10]
    assert o.buffers[got].view(np.int32).tolist() == [0, 1, 2, 3]


def test_nonblocking_allreduce_resolves_the_crossing_deadlock():
    _check_crossing()


def _definitions(n=29):
    """Every rank: iallreduce, ibcast, ireduce, iallgather, then a ring
    isend/irecv, then one waitall over all six requests in another order."""
    R, root = 4, 2
    rng = np.random.default_rng(7)
    b, gs, c = _world(R)
    a = [rng.integers(-2 ** 40, 2 ** 40, n) for _ in range(R)]
    s = [b.buffer(a[r]) for r in range(R)]
    ar = [b.buffer(8 * n) for _ in range(R)]
    bc_data = [rng.integers(-2 ** 31, 2 ** 31, n, dtype=np.int64).astype(np.int32) for _ in range(R)]
    bc = [b.buffer(bc_data[r]) for r in range(R)]
    canary = np.full(8 * n, 0xEE, np.uint8)
    rd = [b.buffer(canary) for _ in range(R)]
    ag_in = [b.buffer(np.full(n, 100 + r, np.int32)) for r in range(R)]
    ag = [b.buffer(4 * n * R) for _ in range(R)]
    ring = [b.buffer(np.full(8, r, np.int32)) for r in range(R)]
    ring_got = [b.buffer(32) for _ in range(R)]
    for r in range(R):
        h1 = b.iallreduce(gs[r], c, s[r], 0, ar[r], 0, n, T_INT64)
        h2 = b.ibcast(gs[r], c, bc[r], 0, n, T_INT32, root)
        h3 = b.ireduce(gs[r], c, s[r], 0, rd[r], 0, n, T_INT64, root, MODE_FIXED)
        h4 = b.iallgather(gs[r], c, ag_in[r], 0, ag[r], 0, n, T_INT32)
        hs = b.isend(gs[r], c, ring[r], 0, 8, T_INT32, (r + 1) % R, 0)
        hr = b.irecv(gs[r], c, ring_got[r], 0, 8, T_INT32, (r - 1) % R, 0)
        b.waitall(gs[r], [h4, hr, h1, hs, h3, h2])
    return b.build(), dict(R=R, n=n, root=root, a=a, ar=ar, bc=bc, bc_data=bc_data, rd=rd,
                           canary=canary, ag=ag, ring_got=ring_got)


def _check_definitions():
    """Each nonblocking kind against its definition, with point-to-point
    traffic between the call and its wait, and waits in a different order."""
    p, m = _definitions()
    R, n, root, a, ar, bc, bc_data, rd, canary, ag, ring_got = (
        m[k] for k in ("R", "n", "root", "a", "ar", "bc", "bc_data", "rd", "canary", "ag", "ring_got"))
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    total = np.sum(np.stack(a), axis=0)  # |values| < 2^40: exact in int64
    for r in range(R):
        assert np.array_equal(o.buffers[ar[r]].view(np.int64), total)
        assert np.array_equal(o.buffers[bc[r]].view(np.int32), bc_data[root])
        if r == root:
            assert np.array_equal(o.buffers[rd[r]].view(np.int64), total)
        else:
            assert np.array_equal(o.buffers[rd[r]], canary)
        want = np.concatenate([np.full(n, 100 + q, np.int32) for q in range(R)])
        assert np.array_equal(o.buffers[ag[r]].view(np.int32), want)
        assert np.all(o.buffers[ring_got[r]].view(np.int32) == (r - 1) % R)


def test_nonblocking_collectives_follow_the_definitions():
    _check_definitions()


def test_blocking_and_nonblocking_share_the_instance_order():
    """Instance k is the k-th collective call of every rank, blocking or not:
    an iallreduce, then a blocking allreduce, on every rank."""
    R, n = 3, 5
    b, gs, c = _world(R)
    xs = [b.buffer(np.full(n, r + 1, np.int64)) for r in range(R)]
    ys = [b.buffer(8 * n) for _ in range(R)]
    zs = [b.buffer(8 * n) for _ in range(R)]
    for r in range(R):
        h = b.iallreduce(gs[r], c, xs[r], 0, ys[r], 0, n, T_INT64)
        b.allreduce(gs[r], c, IN_PLACE, 0, xs[r], 0, n, T_INT64)
        b.wait(gs[r], h)
        b.allreduce(gs[r], c, xs[r], 0, zs[r], 0, n, T_INT64)
    o = oracle.run(b.build())
    assert o.error == 0 and not o.deadlock
    for r in range(R):
        assert np.all(o.buffers[ys[r]].view(np.int64) == 6)
        assert np.all(o.buffers[zs[r]].view(np.int64) == 18)


def test_blocking_and_nonblocking_calls_never_match():
    b, gs, c = _world(2)
    x = [b.buffer(np.ones(4, np.int64)) for _ in range(2)]
    y = [b.buffer(32) for _ in range(2)]
    h = b.iallreduce(gs[0], c, x[0], 0, y[0], 0, 4, T_INT64)
    b.wait(gs[0], h)
    b.allreduce(gs[1], c, x[1], 0, y[1], 0, 4, T_INT64)
    assert oracle.run(b.build()).error != 0


NB_MUTANTS = [
    # a nonblocking collective blocks its stream like the blocking call
    ("              if (is_nonblocking_collective(o.kind)) {  // the stream goes on; a wait completes it",
     "              if (false) {"),
    # the nonblocking reduce computed as an allreduce
    ("    case IREDUCE: return REDUCE;", "    case IREDUCE: return ALLREDUCE;"),
    # the nonblocking bcast computed as an allgather
    ("    case IBCAST: return BCAST;", "    case IBCAST: return ALLGATHER;"),
]


@pytest.mark.parametrize("k", range(len(NB_MUTANTS)))
def test_planted_nonblocking_mistake_is_caught(k, tmp_path, monkeypatch):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "mpx_oracle.cpp")).read()
    old, new = NB_MUTANTS[k]
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
        caught = False
        for fn in (_check_crossing, _check_definitions):
            try:
                fn()
            except AssertionError:
                caught = True
                break
        assert caught, f"mutant {k} survived"
    finally:
        sys.modules["oracle"] = saved
