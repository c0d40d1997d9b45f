"""Pins of the oracle's rooted and gathering collectives against the MPI
definitions restated with numpy: MPI_Bcast (every rank ends with the root's
elements), MPI_Reduce (the root's receive buffer holds the SUM, in rank order
for fp32 fixed mode; other ranks' buffers are untouched), MPI_Allgather
(block s of every receive buffer is rank s's contribution).  Collective calls
on a communicator are ordered: the k-th call of every rank forms instance k,
whatever its kind, and mixing kinds within an instance is an error."""
import numpy as np
import pytest

import oracle
from traffic.program import IN_PLACE, MODE_FIXED, T_FLOAT, T_INT32, T_INT64, ProgramBuilder


def _world(R):
    b = ProgramBuilder(R)
    gs = [b.stream(r) for r in range(R)]
    c = b.comm(gs)
    return b, gs, c


def _vals(rng, n, dt):
    if dt == T_INT64:
        return rng.integers(-2 ** 62, 2 ** 62, n, dtype=np.int64)
    if dt == T_INT32:
        return rng.integers(-2 ** 31, 2 ** 31, n, dtype=np.int64).astype(np.int32)
    return rng.standard_normal(n).astype(np.float32)


@pytest.mark.parametrize("root", [0, 3])
def test_bcast_copies_the_root_everywhere(root):
    R, n = 5, 37
    rng = np.random.default_rng(1)
    b, gs, c = _world(R)
    data = [_vals(rng, n, T_INT32) for _ in range(R)]
    bufs = [b.buffer(d) for d in data]
    for r in range(R):
        b.bcast(gs[r], c, bufs[r], 0, n, T_INT32, root)
    o = oracle.run(b.build())
    assert o.error == 0 and not o.deadlock
    for r in range(R):
        assert np.array_equal(o.buffers[bufs[r]].view(np.int32), data[root])


@pytest.mark.parametrize("dt", [T_INT64, T_FLOAT])
@pytest.mark.parametrize("in_place", [False, True])
def test_reduce_sums_into_the_root_only(dt, in_place):
    R, n, root = 4, 53, 2
    rng = np.random.default_rng(2)
    b, gs, c = _world(R)
    data = [_vals(rng, n, dt) for _ in range(R)]
    npdt = data[0].dtype
    send = [b.buffer(d) for d in data]
    canary = np.full(n * npdt.itemsize, 0xEE, np.uint8)
    recv = [b.buffer(data[r] if (in_place and r == root) else canary) for r in range(R)]
    for r in range(R):
        sb = IN_PLACE if (in_place and r == root) else send[r]
        b.reduce(gs[r], c, sb, 0, recv[r], 0, n, dt, root, MODE_FIXED)
    o = oracle.run(b.build())
    assert o.error == 0 and not o.deadlock
    if dt == T_INT64:
        want = np.array([sum(int(d[i]) for d in data) % (1 << 64) for i in range(n)],
                        np.uint64).view(np.int64)
    else:
        want = data[0].copy()
        for d in data[1:]:
            want = (want + d).astype(np.float32)   # rank order, one rounding per add
    assert np.array_equal(o.buffers[recv[root]].view(npdt), want)
    for r in range(R):
        if r != root:
            assert np.all(o.buffers[recv[r]] == 0xEE), "a non-root receive buffer was written"


@pytest.mark.parametrize("in_place", [False, True])
def test_allgather_concatenates_in_rank_order(in_place):
    R, n = 6, 9
    rng = np.random.default_rng(3)
    b, gs, c = _world(R)
    data = [_vals(rng, n, T_INT64) for _ in range(R)]
    send = [b.buffer(d) for d in data]
    recv = []
    for r in range(R):
        init = np.zeros(R * n, np.int64)
        if in_place:
            init[r * n:(r + 1) * n] = data[r]
        recv.append(b.buffer(init))
    for r in range(R):
        b.allgather(gs[r], c, IN_PLACE if in_place else send[r], 0, recv[r], 0, n, T_INT64)
    o = oracle.run(b.build())
    assert o.error == 0 and not o.deadlock
    want = np.concatenate(data)
    for r in range(R):
        assert np.array_equal(o.buffers[recv[r]].view(np.int64), want)


def test_collective_kinds_share_the_instance_order():
    R, n = 3, 16
    rng = np.random.default_rng(4)
    b, gs, c = _world(R)
    x = [_vals(rng, n, T_INT64) for _ in range(R)]
    xb = [b.buffer(v) for v in x]
    ar = [b.buffer(8 * n) for _ in range(R)]
    ag = [b.buffer(8 * n * R) for _ in range(R)]
    for r in range(R):
        b.allreduce(gs[r], c, xb[r], 0, ar[r], 0, n, T_INT64)
        b.bcast(gs[r], c, ar[r], 0, n, T_INT64, 1)
        b.allgather(gs[r], c, xb[r], 0, ag[r], 0, n, T_INT64)
    o = oracle.run(b.build())
    assert o.error == 0 and not o.deadlock
    total = sum(v.astype(object) for v in x)   # exact; int64 sums wrap modulo 2^64
    for r in range(R):
        assert [int(v) for v in o.buffers[ar[r]].view(np.uint64)] == [int(t) % (1 << 64) for t in total]
        assert np.array_equal(o.buffers[ag[r]].view(np.int64), np.concatenate(x))


def test_mismatched_collective_kinds_are_an_error():
    R, n = 2, 4
    b, gs, c = _world(R)
    x = [b.buffer(np.arange(n, dtype=np.int64)) for _ in range(R)]
    y = [b.buffer(8 * n) for _ in range(R)]
    b.allreduce(gs[0], c, x[0], 0, y[0], 0, n, T_INT64)
    b.bcast(gs[1], c, x[1], 0, n, T_INT64, 0)
    o = oracle.run(b.build())
    assert o.error != 0


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by the pins above
# ---------------------------------------------------------------------------
COLL_MUTANTS = [
    # the broadcast copies rank 0's elements whatever the root
    ("const Op& root = p.ops[arr[(size_t)o0.peer]];", "const Op& root = p.ops[arr[0]];"),
    # the gathered blocks land in reverse rank order
    ("std::memcpy(at(o.buf2, o.off2) + (int64_t)s * bytes, block[s].data(), (size_t)bytes);",
     "std::memcpy(at(o.buf2, o.off2) + (int64_t)s * bytes, block[R - 1 - s].data(), (size_t)bytes);"),
    # an in-place gather takes block 0 of each receive buffer as the contribution
    ("const int64_t so = o.buf == kInPlace ? o.off2 + (int64_t)s * bytes : o.off;",
     "const int64_t so = o.buf == kInPlace ? o.off2 : o.off;"),
    # a reduce writes every rank's receive buffer
    ("const bool writes = root < 0 || (int)k == root;", "const bool writes = true;"),
    # a reduce writes rank 0's receive buffer instead of the root's
    ("const bool writes = root < 0 || (int)k == root;", "const bool writes = root < 0 || k == 0;"),
]


def _collective_checks():
    for root in (0, 3):
        yield lambda root=root: test_bcast_copies_the_root_everywhere(root)
    for dt in (T_INT64, T_FLOAT):
        for in_place in (False, True):
            yield lambda dt=dt, ip=in_place: test_reduce_sums_into_the_root_only(dt, ip)
    for in_place in (False, True):
        yield lambda ip=in_place: test_allgather_concatenates_in_rank_order(ip)
    yield test_collective_kinds_share_the_instance_order


@pytest.mark.parametrize("k", range(len(COLL_MUTANTS)))
def test_planted_collective_mistake_is_caught(k, tmp_path, monkeypatch):
    import importlib
    import os
    import shutil
    import sys
    src = open(os.path.join(os.path.dirname(oracle.__file__), "mpx_oracle.cpp")).read()
    old, new = COLL_MUTANTS[k]
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
        for fn in _collective_checks():
            try:
                fn()
            except AssertionError:
                caught = True
                break
        assert caught, f"mutant {k} survived"
    finally:
        sys.modules["oracle"] = saved
