"""Nonblocking collectives on the GPU path against the oracle, byte for byte:
the crossing pattern that only nonblocking calls complete, every kind with
point-to-point traffic between call and wait (small, vector-aligned and
bulk-copy sizes), a nonblocking barrier, and the argument checks."""
import numpy as np
import pytest

import oracle
from traffic import gen
from tests.test_oracle_nonblocking import _crossing, _definitions
from traffic.program import MODE_FIXED, T_FLOAT, ProgramBuilder

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from traffic import gpu
    return gpu


def _compare(p, mode):
    gpu = _gpu()
    ref = oracle.run(p)
    assert ref.error == 0 and not ref.deadlock
    out = gpu.run(p, mode=mode, timeout_s=60)
    assert out.finished and out.world_error == 0, out.world_error
    for k, (a, b) in enumerate(zip(out.buffers, ref.buffers)):
        assert np.array_equal(a, b), f"buffer {k} differs"
    if p.nstatus:
        assert np.array_equal(out.status, ref.status)


@pytest.mark.parametrize("mode", ["persistent", "drain"])
def test_crossing_pattern_completes(mode):
    p, _, _ = _crossing(True)
    _compare(p, mode)


@pytest.mark.parametrize("n", [29, 4096, 3 << 16])
@pytest.mark.parametrize("mode", ["persistent", "drain"])
def test_every_kind_with_traffic_between_call_and_wait(n, mode):
    p, _ = _definitions(n)
    _compare(p, mode)


def test_fp32_iallreduce_fixed_order_and_ibarrier():
    """fp32 fixed-order sums are bit-exact; a zero-count iallreduce is the
    nonblocking barrier; the stream computes on while both are in flight."""
    R, n = 6, 1 << 18
    rng = np.random.default_rng(11)
    b = ProgramBuilder(R)
    gs = [b.stream(r) for r in range(R)]
    c = b.comm(gs)
    xs = [b.buffer(rng.standard_normal(n).astype(np.float32)) for _ in range(R)]
    ys = [b.buffer(4 * n) for _ in range(R)]
    zs = [b.buffer(np.ones(n, np.float32)) for _ in range(R)]
    ws = [b.buffer(np.full(n, 2.0, np.float32)) for _ in range(R)]
    for r in range(R):
        h = b.iallreduce(gs[r], c, xs[r], 0, ys[r], 0, n, T_FLOAT, MODE_FIXED)
        hb = b.iallreduce(gs[r], c, -1, 0, -1, 0, 0, T_FLOAT)       # ibarrier
        b.axpy(gs[r], 3.0, zs[r], 0, ws[r], 0, n)                    # overlapping compute
        b.waitall(gs[r], [hb, h])
    _compare(b.build(), "persistent")


def test_argument_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_13707_gb300 import mpx
    cfg = mpx.mpx_world_config_init()
    cfg.max_streams = 4
    w = mpx.mpx_world_create(2, cfg)
    raw = [mpx.mpx_cuda_stream_create() for _ in range(2)]
    st = [mpx.mpx_stream_create(w, r, raw[r], mpx.STREAM_DEFAULT) for r in range(2)]
    comm = mpx.mpx_stream_comm_create(w, st)
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    try:
        for fn in (lambda: mpx.mpx_iallreduce_enqueue(p, p, 4, mpx.INT32, 5, comm[0]),
                   lambda: mpx.mpx_ibcast_enqueue(p, 4, mpx.INT32, 2, comm[0]),
                   lambda: mpx.mpx_ireduce_enqueue(p, p, 4, 9, mpx.SUM, 0, comm[0])):
            with pytest.raises(mpx.MpxError) as e:
                fn()
            assert e.value.code in (mpx.ERR_ARG, mpx.ERR_RANK, mpx.ERR_TYPE)
        # a matched nonblocking barrier on both ranks, waited on each stream
        reqs = [mpx.mpx_ibarrier_enqueue(comm[r]) for r in range(2)]
        for q in reqs:
            mpx.mpx_wait_enqueue(q, 0)
        for h in raw:
            torch.cuda.ExternalStream(h).synchronize()
        assert mpx.mpx_world_get_error(w) == 0
    finally:
        for h in comm:
            mpx.mpx_comm_free(h)
        mpx.mpx_world_stop(w, 10000)
        import time
        for s_ in st:
            for _ in range(2000):
                try:
                    mpx.mpx_stream_free(s_)
                    break
                except mpx.MpxError as e:
                    if e.code != mpx.ERR_PENDING:
                        raise
                    time.sleep(5e-4)
        mpx.mpx_world_free(w)
        for h in raw:
            mpx.mpx_cuda_stream_destroy(h)


# ---------------------------------------------------------------------------
# persistent collectives: mpx_*_init once, mpx_start_enqueue per instance
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["persistent", "drain"])
def test_persistent_collectives_match_the_oracle(mode):
    """An in-place int64 allreduce and a broadcast from root 1, each a
    persistent request started three times, with the root's buffer rewritten
    by an axpy between broadcast starts: bit-exact with the oracle."""
    gpu = _gpu()
    p = gen.persistent_collectives(nranks=4, starts=3, n=4099)
    ref = oracle.run(p)
    assert ref.error == 0 and not ref.deadlock
    out = gpu.run(p, mode=mode, timeout_s=45)
    assert out.finished and out.world_error == 0
    for k, (a, b) in enumerate(zip(out.buffers, ref.buffers)):
        assert np.array_equal(a, b), f"buffer {k} differs"


def test_persistent_request_lifecycle():
    """Start of an active request: MPX_ERR_STATE; free while active:
    MPX_ERR_PENDING; a wait leaves the handle valid (startable again); a wait
    on an inactive handle is a no-op; free of an operation's request:
    MPX_ERR_REQUEST; init on the plain path: MPX_ERR_UNSUPPORTED."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_13707_gb300 import mpx
    for mode in (mpx.ENGINE_PERSISTENT, mpx.ENGINE_PLAIN):
        cfg = mpx.mpx_world_config_init()
        cfg.engine_mode = mode
        cfg.max_streams = 4
        w = mpx.mpx_world_create(2, cfg)
        raw = [mpx.mpx_cuda_stream_create() for _ in range(2)]
        cs = [torch.cuda.ExternalStream(h) for h in raw]
        ms = [mpx.mpx_stream_create(w, r, raw[r]) for r in range(2)]
        comm = mpx.mpx_stream_comm_create(w, ms)
        x = torch.arange(8, dtype=torch.int64, device="cuda").repeat(2, 1)
        torch.cuda.synchronize()
        try:
            if mode == mpx.ENGINE_PLAIN:
                with pytest.raises(mpx.MpxError) as e:
                    mpx.mpx_allreduce_init(mpx.IN_PLACE, x[0].data_ptr(), 8, mpx.INT64, mpx.SUM, comm[0])
                assert e.value.code == mpx.ERR_UNSUPPORTED
                continue
            h = [mpx.mpx_allreduce_init(mpx.IN_PLACE, x[r].data_ptr(), 8, mpx.INT64, mpx.SUM, comm[r])
                 for r in range(2)]
            assert all(v not in (-1,) and v < -1 for v in h)
            mpx.mpx_wait_enqueue(h[0])                       # inactive: completes at once
            for rep in range(2):
                for r in range(2):
                    mpx.mpx_start_enqueue(h[r])
                with pytest.raises(mpx.MpxError) as e:
                    mpx.mpx_start_enqueue(h[0])
                assert e.value.code == mpx.ERR_STATE
                with pytest.raises(mpx.MpxError) as e:
                    mpx.mpx_request_free(h[0])
                assert e.value.code == mpx.ERR_PENDING
                for r in range(2):
                    mpx.mpx_wait_enqueue(h[r])
            for s in cs:
                s.synchronize()
            assert x.cpu().tolist() == [[4 * v for v in range(8)]] * 2   # two starts: x*2*2
            q = mpx.mpx_isend_enqueue(x[0].data_ptr(), 1, mpx.INT64, 1, 0, comm[0])
            with pytest.raises(mpx.MpxError) as e:
                mpx.mpx_request_free(q)
            assert e.value.code == mpx.ERR_REQUEST
            r2 = mpx.mpx_irecv_enqueue(x[1].data_ptr(), 1, mpx.INT64, 0, 0, comm[1])
            mpx.mpx_wait_enqueue(q)
            mpx.mpx_wait_enqueue(r2)
            for s in cs:
                s.synchronize()
            for v in h:
                mpx.mpx_request_free(v)
        finally:
            for c in comm:
                mpx.mpx_comm_free(c)
            for s in ms:
                for _ in range(2000):
                    try:
                        mpx.mpx_stream_free(s)
                        break
                    except mpx.MpxError:
                        import time
                        time.sleep(5e-4)
            mpx.mpx_world_free(w)
            for h_ in raw:
                mpx.mpx_cuda_stream_destroy(h_)
