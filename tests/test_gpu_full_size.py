"""Parity at the workloads' full sizes, in the launch configurations the
benchmark times.

* Ring exchange (8 ranks, axpy n = 2^24, messages log-uniform 4 KB - 64 MB,
  half vector-typed): three full-size steps through drain passes, every
  buffer compared byte for byte with the oracle.
* Enqueued allreduce among 16 ranks at n = 2^26 and 2^28 (fp32, fixed and tree
  order) and n = 2^25 and 2^27 (int64): every rank's output must be identical (a
  property at any size), and sampled elements (both ends, tile edges, random
  positions) must equal what the oracle computes for those elements' inputs:
  bit-exact for int64 and the fixed order, within |y - s| <= 1e-6 * sum|x|
  of the oracle's double sum for the tree order.
* One step of the 512^3 halo exchange (8 subdomains of 256^3, six faces
  each, vector-typed x and y faces), every buffer compared with the oracle."""
import numpy as np
import pytest

import oracle
from traffic import gen
from traffic.program import MODE_FIXED, MODE_TREE, T_FLOAT, T_INT64, ProgramBuilder

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def test_ring_exchange_full_size_three_steps():
    _torch()
    from traffic import gpu
    p = gen.ring_exchange(nranks=8, n=1 << 24, steps=3)
    ref = oracle.run(p)
    assert ref.error == 0 and not ref.deadlock
    out = gpu.run(p, mode="drain", timeout_s=120)
    assert out.finished and out.world_error == 0
    for k, (a, b) in enumerate(zip(out.buffers, ref.buffers)):
        assert np.array_equal(a, b), f"buffer {k} differs"


def test_halo_exchange_full_size_step():
    """One step of the 512^3 halo exchange at its full size: 8 subdomains of
    256^3 fp32, each sending its 6 faces (x faces vector(65536, 1, 256) with
    4-byte blocks, y faces vector(256, 256, 65536), z faces contiguous) into
    the neighbours' contiguous ghost buffers; every subdomain and ghost buffer
    compared byte for byte with the oracle."""
    _torch()
    from traffic import gpu
    p = gen.halo3d(sub=256, steps=1)
    ref = oracle.run(p)
    assert ref.error == 0 and not ref.deadlock
    out = gpu.run(p, mode="persistent", timeout_s=120)
    assert out.finished and out.world_error == 0
    for k, (a, b) in enumerate(zip(out.buffers, ref.buffers)):
        assert np.array_equal(a, b), f"buffer {k} differs"


def _sample(n, rng, tile=8192, m=4096):
    edges = np.arange(tile, n, tile)
    idx = np.concatenate([[0, 1, n - 2, n - 1], edges[:512] - 1, edges[:512],
                          rng.integers(0, n, m)])
    return np.unique(idx[(idx >= 0) & (idx < n)])


def _oracle_allreduce(cols, dt, mode):
    """Oracle result for one allreduce whose rank r contributes cols[r]."""
    R, m = cols.shape
    b = ProgramBuilder(R, "allreduce-sample")
    gs = [b.stream(r) for r in range(R)]
    c = b.comm(gs)
    for r in range(R):
        sb = b.buffer(cols[r])
        rb = b.buffer(cols[r].nbytes)
        b.allreduce(gs[r], c, sb, 0, rb, 0, m, dt, mode)
    p = b.build()
    o = oracle.run(p)
    assert o.error == 0 and not o.deadlock
    return [o.buffers[2 * r + 1].view(cols.dtype) for r in range(R)]


@pytest.mark.parametrize("dt_name,lg,mode", [("f32", 26, "fixed"), ("f32", 26, "tree"),
                                             ("int64", 25, "fixed"), ("f32", 28, "fixed"),
                                             ("int64", 27, "fixed")])
def test_allreduce_full_size_sampled(dt_name, lg, mode):
    torch = _torch()
    from paper_2208_13707_gb300 import mpx
    R, n = 16, 1 << lg
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(0x220813707 + 3)
    if dt_name == "f32":
        x = torch.randn((R, n), device=dev, generator=g, dtype=torch.float32)
        dt, tdt, npdt = mpx.FLOAT, T_FLOAT, np.float32
    else:
        x = torch.empty((R, n), device=dev, dtype=torch.int64)
        for r in range(R):  # one rank at a time: small temporaries at 2^27 elements
            x[r].copy_(torch.round(torch.randn(n, device=dev, generator=g) * 2.0 ** 40).to(torch.int64))
        dt, tdt, npdt = mpx.INT64, T_INT64, np.int64
    y = torch.zeros_like(x)
    cfg = mpx.mpx_world_config_init()
    cfg.max_streams = R
    world = mpx.mpx_world_create(R, cfg)
    raw = [mpx.mpx_cuda_stream_create() for _ in range(R)]
    cs = [torch.cuda.ExternalStream(h, device=dev) for h in raw]
    ms = [mpx.mpx_stream_create(world, r, raw[r], mpx.STREAM_EXCLUSIVE) for r in range(R)]
    comm = mpx.mpx_stream_comm_create(world, ms)
    m_ = mpx.REDUCE_TREE if mode == "tree" else mpx.REDUCE_FIXED
    mpx.mpx_comm_set_reduce_mode(comm[0], m_)
    torch.cuda.synchronize()
    try:
        for r in range(R):
            mpx.mpx_allreduce_enqueue(x[r].data_ptr(), y[r].data_ptr(), n, dt, mpx.SUM, comm[r])
        for c in cs:
            c.synchronize()
        assert mpx.mpx_world_get_error(world) == 0
        for r in range(1, R):
            assert torch.equal(y[0], y[r]), f"rank {r} output differs from rank 0"
        idx = _sample(n, np.random.default_rng(lg))
        ti = torch.from_numpy(idx).to(dev)
        cols = x[:, ti].cpu().numpy().astype(npdt)
        got = y[0, ti].cpu().numpy()
        if mode == "tree":
            s, a = oracle.sum_f32_ref([cols[r] for r in range(R)])
            err = np.abs(got.astype(np.float64) - s)
            assert np.all(err <= 1e-6 * a), f"max err/bound {np.max(err / np.maximum(a, 1e-300))}"
        else:
            want = _oracle_allreduce(cols, tdt, MODE_FIXED)[0]
            assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), "sampled outputs differ"
        mpx.mpx_world_stop(world, 10000)
    finally:
        for h in comm:
            mpx.mpx_comm_free(h)
        for s_ in ms:
            mpx.mpx_stream_free(s_)
        mpx.mpx_world_free(world)
        for h in raw:
            mpx.mpx_cuda_stream_destroy(h)


def test_batching_full_size_epoch():
    """One epoch of the batching configuration at full message sizes: 64
    ranks x 4 MPIX streams, 65,536 messages of 8 B - 1 MB with ANY_TAG and
    ANY_SOURCE receives, through the persistent engine with batch submission
    (the launch configuration the benchmark times).  Every status and the
    receive buffers of a sample of streams are compared with the oracle."""
    _torch()
    from traffic import gpu
    p = gen.batching(nranks=64, streams_per_rank=4, nmsg=65536, max_bytes=1 << 20,
                     laminar=True, seed=gen.SEED_BASE + 2)
    ref = oracle.run(p)
    assert ref.error == 0 and not ref.deadlock
    r = gpu.BatchRunner(p, mode="persistent", timeout_s=120,
                        cfg_over={"ring_slots": 4096, "queue_slots": 4096})
    try:
        assert r.step(), "epoch did not finish"
        serr, werr = r.errors()
        assert werr == 0 and not any(serr)
        st = np.frombuffer(r.st.cpu().numpy().tobytes(), ref.status.dtype)[: p.nstatus]
        assert np.array_equal(st, ref.status), "statuses differ"
        rng = np.random.default_rng(7)
        nbuf = len(p.buf_init)
        for k in sorted(rng.choice(nbuf, size=24, replace=False)):
            got = r.dbufs[k].cpu().numpy()[: p.buf_init[k].size]
            assert np.array_equal(got, ref.buffers[k]), f"buffer {k} differs"
    finally:
        r.close()
