"""mpx_sendrecv_static: the staged copy that allocates nothing, for callers
that cannot call cudaMalloc (inside a stream capture, on paths that must not
synchronize the device, in processes with pre-partitioned device memory).

Its output must equal what the engine's send/receive path delivers for the
same layouts, byte for byte, on two calls in a row (the calls share the one
static staging array).  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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
                import time
                time.sleep(5e-4)
    mpx.mpx_world_free(w)
    for h in raw:
        mpx.mpx_cuda_stream_destroy(h)
    return out


def test_sendrecv_static_matches_engine_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_13707_gb300 import mpx
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(2208)
    src = torch.randint(0, 256, (3 << 20,), generator=g, device=dev, dtype=torch.uint8)
    dst_init = torch.randint(0, 256, (3 << 20,), generator=g, device=dev, dtype=torch.uint8)
    vec = mpx.mpx_type_vector(4000, 64, 128, mpx.FLOAT)       # 1 MiB of data, 2 MiB extent
    cases = [
        # vector -> contiguous, receive shorter than the message (truncation)
        (1, vec, 200_000, mpx.FLOAT),
        # contiguous -> vector
        (256_000, mpx.FLOAT, 1, vec),
    ]
    raw = mpx.mpx_cuda_stream_create()
    stream = torch.cuda.ExternalStream(raw)
    try:
        for s_cnt, s_ty, r_cnt, r_ty in cases:          # two calls in a row
            ref = _engine_reference(mpx, torch, src, dst_init, s_cnt, s_ty, r_cnt, r_ty)
            dst = dst_init.clone()
            torch.cuda.synchronize()
            n = mpx.mpx_sendrecv_static(src.data_ptr(), s_cnt, s_ty, dst.data_ptr(), r_cnt, r_ty, raw)
            stream.synchronize()
            got = dst.cpu().numpy()
            assert n == min(s_cnt * mpx.mpx_type_size(s_ty), r_cnt * mpx.mpx_type_size(r_ty))
            assert np.array_equal(got, ref)
        # beyond the static area: a clear error, nothing enqueued
        with pytest.raises(mpx.MpxError) as e:
            mpx.mpx_sendrecv_static(src.data_ptr(), (17 << 20) // 4, mpx.FLOAT, dst.data_ptr(),
                                    (17 << 20) // 4, mpx.FLOAT, raw)
        assert e.value.code == mpx.ERR_NO_MEM
    finally:
        mpx.mpx_type_free(vec)
        mpx.mpx_cuda_stream_destroy(raw)
