"""Enqueued bcast, reduce, allgather and barrier on the GPU against the
oracle, byte for byte (fp32 tree-order reductions within the stated bound):
unaligned counts (element path), aligned ones (16-byte vectors) and large
ones (bulk copies through shared memory), roots other than 0, in-place
forms, and mixed sequences on one communicator."""
import numpy as np
import pytest

import oracle
from traffic.program import (IN_PLACE, MODE_FIXED, MODE_TREE, T_BYTE, T_FLOAT, T_INT32, T_INT64,
                             ProgramBuilder)

pytestmark = pytest.mark.gpu

NP = {T_BYTE: np.uint8, T_INT32: np.int32, T_INT64: np.int64, T_FLOAT: np.float32}


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from traffic import gpu
    return gpu


def _vals(rng, n, dt):
    if dt == T_FLOAT:
        return rng.standard_normal(n).astype(np.float32)
    info = np.iinfo(NP[dt])
    return rng.integers(info.min, info.max, n, dtype=np.int64).astype(NP[dt])


def _run(p, mode="persistent", exact_bufs=None):
    gpu = _gpu()
    ref = oracle.run(p)
    assert ref.error == 0 and not ref.deadlock
    out = gpu.run(p, mode=mode, timeout_s=60)
    assert out.finished and out.world_error == 0, out.world_error
    for k, (a, b) in enumerate(zip(out.buffers, ref.buffers)):
        if exact_bufs is None or k in exact_bufs:
            assert np.array_equal(a, b), f"buffer {k} differs"
    return out, ref


@pytest.mark.parametrize("n", [37, 4103, 1 << 20])
@pytest.mark.parametrize("root", [0, 3])
def test_bcast(n, root):
    R = 5
    rng = np.random.default_rng(n + root)
    b = ProgramBuilder(R)
    gs = [b.stream(r) for r in range(R)]
    c = b.comm(gs)
    bufs = [b.buffer(_vals(rng, n, T_INT32)) for _ in range(R)]
    for r in range(R):
        b.bcast(gs[r], c, bufs[r], 0, n, T_INT32, root)
    _run(b.build())


@pytest.mark.parametrize("dt,n", [(T_INT64, 1001), (T_FLOAT, 4096), (T_FLOAT, 3 << 18),
                                  (T_BYTE, 77)])
@pytest.mark.parametrize("in_place", [False, True])
def test_reduce_fixed(dt, n, in_place):
    R, root = 6, 4
    rng = np.random.default_rng(n)
    b = ProgramBuilder(R)
    gs = [b.stream(r) for r in range(R)]
    c = b.comm(gs)
    data = [_vals(rng, n, dt) for _ in range(R)]
    send = [b.buffer(d) for d in data]
    recv = [b.buffer(data[r] if (in_place and r == root) else np.full(n * data[0].itemsize, 0xEE, np.uint8))
            for r in range(R)]
    for r in range(R):
        sb = IN_PLACE if (in_place and r == root) else send[r]
        b.reduce(gs[r], c, sb, 0, recv[r], 0, n, dt, root, MODE_FIXED)
    _run(b.build())


def test_reduce_tree_within_bound():
    R, root, n = 16, 7, 1 << 20
    rng = np.random.default_rng(11)
    b = ProgramBuilder(R)
    gs = [b.stream(r) for r in range(R)]
    c = b.comm(gs)
    data = [rng.standard_normal(n).astype(np.float32) for _ in range(R)]
    send = [b.buffer(d) for d in data]
    recv = [b.buffer(4 * n) for _ in range(R)]
    for r in range(R):
        b.reduce(gs[r], c, send[r], 0, recv[r], 0, n, T_FLOAT, root, MODE_TREE)
    p = b.build()
    out, ref = _run(p, exact_bufs=set(send))
    got = out.buffers[recv[root]].view(np.float32).astype(np.float64)
    s, a = oracle.sum_f32_ref(data)
    assert np.all(np.abs(got - s) <= 1e-6 * a)
    for r in range(R):
        if r != root:
            assert np.all(out.buffers[recv[r]] == 0)


@pytest.mark.parametrize("dt,n", [(T_INT64, 9), (T_FLOAT, 1024), (T_FLOAT, 1 << 18), (T_BYTE, 33)])
@pytest.mark.parametrize("in_place", [False, True])
def test_allgather(dt, n, in_place):
    R = 5
    rng = np.random.default_rng(n + 1)
    b = ProgramBuilder(R)
    gs = [b.stream(r) for r in range(R)]
    c = b.comm(gs)
    data = [_vals(rng, n, dt) for _ in range(R)]
    send = [b.buffer(d) for d in data]
    recv = []
    for r in range(R):
        init = np.zeros(R * n, NP[dt])
        if in_place:
            init[r * n:(r + 1) * n] = data[r]
        recv.append(b.buffer(init))
    for r in range(R):
        b.allgather(gs[r], c, IN_PLACE if in_place else send[r], 0, recv[r], 0, n, dt)
    _run(b.build())


@pytest.mark.parametrize("mode", ["persistent", "drain"])
def test_mixed_collectives_and_p2p(mode):
    """allreduce, barrier (an allreduce of no elements), bcast from the
    allreduce's result, allgather and a ring of isend/irecv on one
    communicator, in the same order on every rank."""
    R, n = 4, 3000
    rng = np.random.default_rng(5)
    b = ProgramBuilder(R)
    gs = [b.stream(r) for r in range(R)]
    c = b.comm(gs)
    x = [b.buffer(_vals(rng, n, T_INT64)) for _ in range(R)]
    ar = [b.buffer(8 * n) for _ in range(R)]
    ag = [b.buffer(8 * n * R) for _ in range(R)]
    rb = [b.buffer(8 * n) for _ in range(R)]
    for r in range(R):
        b.allreduce(gs[r], c, x[r], 0, ar[r], 0, n, T_INT64)
        b.allreduce(gs[r], c, -1, 0, -1, 0, 0, T_INT64)  # barrier
        b.bcast(gs[r], c, ar[r], 0, n, T_INT64, 2)
        b.allgather(gs[r], c, x[r], 0, ag[r], 0, n, T_INT64)
        h1 = b.isend(gs[r], c, ag[r], 8 * n * r, n, T_INT64, (r + 1) % R, 9)
        h2 = b.irecv(gs[r], c, rb[r], 0, n, T_INT64, (r - 1) % R, 9)
        b.waitall(gs[r], [h1, h2])
    _run(b.build(), mode=mode)
