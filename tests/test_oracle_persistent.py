"""Pins for persistent collectives in the oracle (MPI-4: a persistent
collective started by MPI_Start behaves as the nonblocking collective with
the recorded arguments, initiated at the start).  The oracle runs each start
as that nonblocking call; these tests check it against closed forms: an
in-place int64 allreduce started k times leaves R^(k-1) * sum of the
initial values on every rank (two's-complement wrap), and a broadcast start
delivers the root's buffer as it stands when the root's stream reaches the
start (after the axpys before it)."""
import numpy as np

import oracle
from traffic import gen
from traffic.program import IALLREDUCE, IBCAST, WAIT


def _wrap(v):
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >= 1 << 63 else v


def test_persistent_allreduce_started_k_times_closed_form():
    for R, k in ((4, 3), (3, 5)):
        p = gen.persistent_collectives(nranks=R, starts=k, n=257)
        o = oracle.run(p)
        assert o.error == 0 and not o.deadlock
        Y0 = [p.buf_init[y].view(np.int64) for y in p.meta["Y"]]
        for i in (0, 1, 128, 256):
            s = sum(int(y[i]) for y in Y0)
            want = _wrap(R ** (k - 1) * s)
            for r in range(R):
                assert int(o.buffers[p.meta["Y"][r]].view(np.int64)[i]) == want


def test_persistent_bcast_reads_the_root_buffer_at_each_start():
    p = gen.persistent_collectives(nranks=4, starts=3, n=64)
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    X = p.buf_init[p.meta["X"][1]].view(np.float32)
    b = p.buf_init[p.meta["B"][1]].view(np.float32).copy()
    for _ in range(3):   # the root's axpy (single rounding), then the broadcast of its B
        b = (0.5 * X.astype(np.float64) + b.astype(np.float64)).astype(np.float32)
    for r in range(4):
        assert np.array_equal(o.buffers[p.meta["B"][r]].view(np.float32), b)


def test_starts_are_the_nonblocking_calls_in_the_program():
    """The program marks every start with its persistent request; each start
    is followed by a wait on it, and every rank starts in the same order."""
    p = gen.persistent_collectives(nranks=3, starts=2, n=8)
    ops = p.ops
    starts = ops[ops["persist"] > 0]
    assert set(int(k) for k in starts["kind"]) == {IALLREDUCE, IBCAST}
    assert np.sum(ops["kind"] == WAIT) == len(starts)
    per = [list(starts[starts["stream"] == g]["kind"]) for g in range(3)]
    assert per[0] == per[1] == per[2]
