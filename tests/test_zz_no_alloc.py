"""mpx_sendrecv_static: the staged copy that allocates nothing, for callers
that cannot call cudaMalloc (paths that must not risk a device-wide
synchronization, processes whose device memory is carved up in advance).

Its output must equal what the engine's send/receive path delivers for the
same layouts, byte for byte, on two calls in a row (the calls share the one
static staging array), and must equal MPI_Type_vector packing and unpacking
restated as 2-D array slices (tests/checks.py, independent of both CUDA
paths).  It must also run while a persistent engine is resident: its kernel
and its array's address are set up when a world is created, so its first
launch never waits for the engine to leave.  This file is collected last on
purpose."""
import time

import numpy as np
import pytest

from checks import np_pack, np_unpack
from traffic.program import TYPE_DTYPE, basic_types

pytestmark = pytest.mark.gpu


def _types_table(mpx, vec_shape):
    """The program-style type table (ids 0..4 predefined, 5 = the vector)."""
    t = np.concatenate([basic_types(), np.zeros(1, TYPE_DTYPE)])
    vc, bl, st = vec_shape
    t[5] = (1, mpx.FLOAT, 4, vc, bl, st)
    return t


def _expected(src, dst_init, s_cnt, s_id, r_cnt, r_id, table):
    """MPI's answer: pack the send side, deliver min(sent, capacity) bytes."""
    packed = np_pack(src, 0, table, s_id, s_cnt)
    cap = len(np_pack(dst_init, 0, table, r_id, r_cnt))
    out = dst_init.copy()
    np_unpack(out, 0, table, r_id, r_cnt, packed[: min(len(packed), cap)])
    return out


def _engine_reference(mpx, torch, src, dst_init, s_cnt, s_ty, r_cnt, r_ty):
    """Deliver through the existing entry points: send_enqueue / recv_enqueue."""
    cfg = mpx.mpx_world_config_init()
    cfg.max_streams = 4
    w = mpx.mpx_world_create(2, cfg)
    raw = [mpx.mpx_cuda_stream_create() for _ in range(2)]
    cs = [torch.cuda.ExternalStream(h) for h in raw]
    ms = [mpx.mpx_stream_create(w, r, raw[r]) for r in range(2)]
    comm = mpx.mpx_stream_comm_create(w, ms)
    dst = dst_init.clone()
    torch.cuda.synchronize()
    mpx.mpx_send_enqueue(src.data_ptr(), s_cnt, s_ty, 1, 7, comm[0])
    mpx.mpx_recv_enqueue(dst.data_ptr(), r_cnt, r_ty, 0, 7, comm[1])
    for s in cs:
        s.synchronize()
    out = dst.cpu().numpy().copy()
    for c in comm:
        mpx.mpx_comm_free(c)
    for s in ms:
        for _ in range(2000):
            try:
                mpx.mpx_stream_free(s)
                break
            except mpx.MpxError:
                time.sleep(5e-4)
    mpx.mpx_world_free(w)
    for h in raw:
        mpx.mpx_cuda_stream_destroy(h)
    return out


def _setup(torch, mpx):
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(2208)
    src = torch.randint(0, 256, (3 << 20,), generator=g, device=dev, dtype=torch.uint8)
    dst_init = torch.randint(0, 256, (3 << 20,), generator=g, device=dev, dtype=torch.uint8)
    return src, dst_init


def test_sendrecv_static_matches_engine_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_13707_gb300 import mpx
    src, dst_init = _setup(torch, mpx)
    shape = (4000, 64, 128)
    vec = mpx.mpx_type_vector(*shape, mpx.FLOAT)            # 1 MiB of data, 2 MiB extent
    table = _types_table(mpx, shape)
    cases = [
        # vector -> contiguous, receive shorter than the message (truncation)
        (1, (vec, 5), 200_000, (mpx.FLOAT, mpx.FLOAT)),
        # contiguous -> vector
        (256_000, (mpx.FLOAT, mpx.FLOAT), 1, (vec, 5)),
    ]
    src_np, dst_np = src.cpu().numpy(), dst_init.cpu().numpy()
    raw = mpx.mpx_cuda_stream_create()
    stream = torch.cuda.ExternalStream(raw)
    try:
        for s_cnt, (s_ty, s_id), r_cnt, (r_ty, r_id) in cases:    # two calls in a row
            ref = _engine_reference(mpx, torch, src, dst_init, s_cnt, s_ty, r_cnt, r_ty)
            want = _expected(src_np, dst_np, s_cnt, s_id, r_cnt, r_id, table)
            dst = dst_init.clone()
            torch.cuda.synchronize()
            n = mpx.mpx_sendrecv_static(src.data_ptr(), s_cnt, s_ty, dst.data_ptr(), r_cnt, r_ty, raw)
            stream.synchronize()
            got = dst.cpu().numpy()
            assert n == min(s_cnt * mpx.mpx_type_size(s_ty), r_cnt * mpx.mpx_type_size(r_ty))
            assert np.array_equal(got, ref), "differs from the engine's send/receive"
            assert np.array_equal(got, want), "differs from MPI_Type_vector packing"
        # beyond the static area: a clear error, nothing enqueued
        with pytest.raises(mpx.MpxError) as e:
            mpx.mpx_sendrecv_static(src.data_ptr(), (17 << 20) // 4, mpx.FLOAT, dst.data_ptr(),
                                    (17 << 20) // 4, mpx.FLOAT, raw)
        assert e.value.code == mpx.ERR_NO_MEM
    finally:
        mpx.mpx_type_free(vec)
        mpx.mpx_cuda_stream_destroy(raw)


def test_sendrecv_static_next_to_a_resident_engine():
    """A persistent engine kept resident by a receive that is not yet matched;
    meanwhile the static copy runs on another stream and finishes well before
    the engine's watchdog; then the receive's send completes the world's work."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_13707_gb300 import mpx
    src, dst_init = _setup(torch, mpx)
    cfg = mpx.mpx_world_config_init()
    cfg.engine_mode = mpx.ENGINE_PERSISTENT
    cfg.max_streams = 4
    cfg.watchdog_ns = int(20e9)
    w = mpx.mpx_world_create(2, cfg)
    raw = [mpx.mpx_cuda_stream_create() for _ in range(3)]
    cs = [torch.cuda.ExternalStream(h) for h in raw]
    ms = [mpx.mpx_stream_create(w, r, raw[r]) for r in range(2)]
    comm = mpx.mpx_stream_comm_create(w, ms)
    box = torch.zeros(64, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    try:
        req = mpx.mpx_irecv_enqueue(box.data_ptr(), 64, mpx.BYTE, 0, 3, comm[1])
        time.sleep(0.01)                       # the engine is resident, the receive pending
        dst = dst_init.clone()
        # (a device-wide synchronize would wait for the resident engine itself)
        torch.cuda.current_stream().synchronize()
        t0 = time.perf_counter()
        n = mpx.mpx_sendrecv_static(src.data_ptr(), 1 << 18, mpx.FLOAT, dst.data_ptr(), 1 << 18,
                                    mpx.FLOAT, raw[2])
        cs[2].synchronize()
        dt = time.perf_counter() - t0
        assert n == 1 << 20
        assert np.array_equal(dst.cpu().numpy()[: 1 << 20], src.cpu().numpy()[: 1 << 20])
        assert dt < 5.0, f"static copy waited {dt:.1f} s behind the resident engine"
        assert mpx.mpx_world_get_error(w) == 0
        mpx.mpx_send_enqueue(src.data_ptr(), 64, mpx.BYTE, 1, 3, comm[0])
        mpx.mpx_wait_enqueue(req)
        for s in cs[:2]:
            s.synchronize()
        assert np.array_equal(box.cpu().numpy(), src.cpu().numpy()[:64])
    finally:
        for c in comm:
            mpx.mpx_comm_free(c)
        for s in ms:
            for _ in range(2000):
                try:
                    mpx.mpx_stream_free(s)
                    break
                except mpx.MpxError:
                    time.sleep(5e-4)
        mpx.mpx_world_free(w)
        for h in raw:
            mpx.mpx_cuda_stream_destroy(h)
