"""Unit checks on the GPU for the edges of the copy path and the limits of the
enqueue path: every byte offset of source and destination through the 16-byte
vector and the bulk-copy paths, compared with the oracle byte for byte; a full
submission ring; a stream freed with work in flight; a world larger than its
device budget.  No test faults or hangs the GPU: the limits come back as the
library's error codes, and a receive nobody sends is released by
mpx_world_abort."""
import time

import numpy as np
import pytest

import oracle
from traffic.program import T_BYTE, ProgramBuilder

pytestmark = pytest.mark.gpu


def _env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_13707_gb300 import mpx
    return torch, mpx


def _offsets_program():
    """Rank 0 sends, rank 1 receives, one message per (size, source offset,
    destination offset): every source offset 0..15 with a permutation of the
    destination offsets for each size, and every pair of offsets at 4099 bytes.
    Sizes from 1 byte to several tiles, around the bulk-copy threshold."""
    rng = np.random.default_rng(0x220813707 + 11)
    cases = []
    for size in (1, 15, 17, 4099, (40 << 10) + 5, (300 << 10) + 11):
        for s in range(16):
            cases.append((size, s, (7 * s + size) % 16))
    cases += [(4099, s, d) for s in range(16) for d in range(16)]
    span = [((n + 16 + 255) // 256) * 256 for n, _, _ in cases]
    base = np.concatenate([[0], np.cumsum(span)[:-1]]).astype(np.int64)
    total = int(sum(span))
    b = ProgramBuilder(2, "byte-offsets")
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    src = b.buffer(rng.integers(0, 256, total, dtype=np.uint8))
    dst = b.buffer(total)
    sends, recvs = [], []
    for k, ((n, so, do), at) in enumerate(zip(cases, base)):
        sends.append(b.isend(g0, c, src, int(at) + so, n, T_BYTE, 1, k))
        recvs.append(b.irecv(g1, c, dst, int(at) + do, n, T_BYTE, 0, k))
    b.waitall(g0, sends)
    b.waitall(g1, recvs)
    return b.build()


@pytest.mark.parametrize("cfg_over", [
    {},                                                 # 64 KiB tiles, bulk copies from 32 KiB
    {"tile_bytes": 4096},                               # small tiles: the 16-byte vector path
    {"tile_bytes": 16384, "bulk_min_bytes": 4096},      # bulk copies for tiles from 4 KiB
], ids=["default", "vector_tiles", "bulk_tiles"])
@pytest.mark.parametrize("mode", ["drain", "persistent"])
def test_copies_at_every_byte_offset(mode, cfg_over):
    _env()
    from traffic import gpu
    p = _offsets_program()
    ref = oracle.run(p)
    assert ref.error == 0 and not ref.deadlock
    out = gpu.run(p, mode=mode, cfg_over=cfg_over, timeout_s=60)
    assert out.finished and out.world_error == 0
    for k, (a, b) in enumerate(zip(out.buffers, ref.buffers)):
        if not np.array_equal(a, b):
            diff = np.nonzero(a != b)[0]
            raise AssertionError(f"buffer {k}: {len(diff)} bytes differ, first at {diff[:8]}")


def _world(mpx, torch, **over):
    cfg = mpx.mpx_world_config_init()
    cfg.engine_mode = mpx.ENGINE_PERSISTENT
    cfg.watchdog_ns = int(60e9)
    for k, v in over.items():
        setattr(cfg, k, v)
    w = mpx.mpx_world_create(2, cfg)
    raw = [mpx.mpx_cuda_stream_create() for _ in range(2)]
    cs = [torch.cuda.ExternalStream(h) for h in raw]
    ms = [mpx.mpx_stream_create(w, r, raw[r], mpx.STREAM_EXCLUSIVE) for r in range(2)]
    comm = mpx.mpx_stream_comm_create(w, ms)
    return w, raw, cs, ms, comm


def _release_and_free(mpx, w, raw, cs, ms, comm):
    """Abort releases whatever waits; then everything is freed in order."""
    mpx.mpx_world_abort(w)
    t_dl = time.perf_counter() + 10.0
    while not all(c.query() for c in cs) and time.perf_counter() < t_dl:
        time.sleep(1e-3)
    for c in comm:
        mpx.mpx_comm_free(c)
    t_dl = time.perf_counter() + 10.0
    while any(mpx.mpx_stream_pending(s) for s in ms) and time.perf_counter() < t_dl:
        time.sleep(1e-3)
    for s in ms:
        mpx.mpx_stream_free(s)
    mpx.mpx_world_free(w)
    for h in raw:
        mpx.mpx_cuda_stream_destroy(h)


def test_full_submission_ring_returns_again():
    """A ring of 16 slots holding 16 receives nobody sends (never retired):
    the 17th enqueue waits for a slot for a bounded time, then returns
    MPX_ERR_AGAIN with nothing enqueued."""
    torch, mpx = _env()
    w, raw, cs, ms, comm = _world(mpx, torch, ring_slots=16)
    buf = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    try:
        for k in range(16):
            mpx.mpx_irecv_enqueue(buf.data_ptr() + 64 * k, 8, mpx.BYTE, 0, k, comm[1])
        t0 = time.perf_counter()
        with pytest.raises(mpx.MpxError) as e:
            mpx.mpx_irecv_enqueue(buf.data_ptr(), 8, mpx.BYTE, 0, 99, comm[1])
        assert e.value.code == mpx.ERR_AGAIN
        assert time.perf_counter() - t0 < 10.0
        assert mpx.mpx_stream_pending(ms[1]) == 16
    finally:
        _release_and_free(mpx, w, raw, cs, ms, comm)


def test_stream_free_with_work_in_flight_is_refused():
    """MPIX_Stream_free fails while operations are pending on the stream (§3.1)."""
    torch, mpx = _env()
    w, raw, cs, ms, comm = _world(mpx, torch)
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    try:
        mpx.mpx_irecv_enqueue(buf.data_ptr(), 8, mpx.BYTE, 0, 5, comm[1])
        with pytest.raises(mpx.MpxError) as e:
            mpx.mpx_stream_free(ms[1])
        assert e.value.code == mpx.ERR_PENDING
    finally:
        _release_and_free(mpx, w, raw, cs, ms, comm)


def test_world_beyond_its_device_budget_is_refused():
    _, mpx = _env()
    cfg = mpx.mpx_world_config_init()
    cfg.budget_bytes = 1 << 20  # less than the staging arena alone
    with pytest.raises(mpx.MpxError) as e:
        mpx.mpx_world_create(2, cfg)
    assert e.value.code == mpx.ERR_NO_MEM
