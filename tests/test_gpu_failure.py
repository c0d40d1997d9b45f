"""Failure detection without a GPU fault: every device-side wait is bounded.
A receive that nothing will ever match is the failure here; the engine's
watchdog, or mpx_world_abort from the host, must release the waiting CUDA
stream with MPX_ERR_TIMEOUT in the status and the sticky errors, and the
world must refuse further work.  No test faults, traps or hangs the GPU: the
waits end through the library's own bounded paths."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_13707_gb300 import mpx
    return torch, mpx


def _world(mpx, torch, mode, watchdog_ns):
    cfg = mpx.mpx_world_config_init()
    cfg.engine_mode = mode
    cfg.watchdog_ns = int(watchdog_ns)
    w = mpx.mpx_world_create(2, cfg)
    raw = [mpx.mpx_cuda_stream_create() for _ in range(3)]
    cs = [torch.cuda.ExternalStream(h) for h in raw]
    ms = [mpx.mpx_stream_create(w, r, raw[r], mpx.STREAM_EXCLUSIVE) for r in range(2)]
    comm = mpx.mpx_stream_comm_create(w, ms)
    return w, raw, cs, ms, comm


def _teardown(mpx, w, raw, ms, comm, cs=None):
    if cs is not None and not all(c.query() for c in cs):
        mpx.mpx_world_abort(w)  # never leave a stream waiting
        for c in cs:
            _wait_idle(c, 10.0)
    for c in comm:
        mpx.mpx_comm_free(c)
    # the engine retires released operations shortly after they were released
    t_dl = time.perf_counter() + 10.0
    while any(mpx.mpx_stream_pending(s) for s in ms) and time.perf_counter() < t_dl:
        time.sleep(1e-3)
    for s in ms:
        mpx.mpx_stream_free(s)
    mpx.mpx_world_free(w)
    for h in raw:
        mpx.mpx_cuda_stream_destroy(h)


def _wait_idle(stream, seconds):
    t_dl = time.perf_counter() + seconds
    while not stream.query():
        if time.perf_counter() > t_dl:
            return False
        time.sleep(1e-3)
    return True


def _status(torch, st):
    from traffic.program import STATUS_DTYPE
    return np.frombuffer(st.cpu().numpy().tobytes(), STATUS_DTYPE)[0]


def test_watchdog_releases_a_receive_nobody_sends():
    torch, mpx = _env()
    w, raw, cs, ms, comm = _world(mpx, torch, mpx.ENGINE_PERSISTENT, 0.3e9)
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st = torch.zeros(24, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    try:
        mpx.mpx_recv_enqueue(buf.data_ptr(), 16, mpx.BYTE, 0, 5, comm[1], st.data_ptr())
        assert _wait_idle(cs[1], 20.0), "the watchdog did not release the stream"
        assert _status(torch, st)["error"] == mpx.ERR_TIMEOUT
        assert mpx.mpx_world_get_error(w) == mpx.ERR_TIMEOUT
        assert mpx.mpx_stream_get_error(ms[1]) == mpx.ERR_TIMEOUT
        with pytest.raises(mpx.MpxError) as e:
            mpx.mpx_send_enqueue(buf.data_ptr(), 16, mpx.BYTE, 1, 5, comm[0])
        assert e.value.code == mpx.ERR_STATE
        assert np.all(buf.cpu().numpy() == 0), "a released receive moved data"
    finally:
        _teardown(mpx, w, raw, ms, comm, cs)


def test_host_abort_releases_waiting_streams():
    torch, mpx = _env()
    w, raw, cs, ms, comm = _world(mpx, torch, mpx.ENGINE_PERSISTENT, 60e9)
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st = torch.zeros(24, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    try:
        mpx.mpx_recv_enqueue(buf.data_ptr(), 16, mpx.BYTE, 0, 7, comm[1], st.data_ptr())
        time.sleep(0.05)
        assert not cs[1].query(), "the receive completed without a sender"
        mpx.mpx_world_abort(w)
        assert _wait_idle(cs[1], 10.0), "abort did not release the stream"
        assert mpx.mpx_world_get_error(w) == mpx.ERR_TIMEOUT
        # the resident engine writes the released receive's status
        t_dl = time.perf_counter() + 10.0
        while _status(torch, st)["error"] != mpx.ERR_TIMEOUT and time.perf_counter() < t_dl:
            time.sleep(1e-3)
        assert _status(torch, st)["error"] == mpx.ERR_TIMEOUT
    finally:
        _teardown(mpx, w, raw, ms, comm, cs)


def test_drain_pass_returns_with_an_unmatched_receive():
    torch, mpx = _env()
    w, raw, cs, ms, comm = _world(mpx, torch, mpx.ENGINE_DRAIN, 60e9)
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    try:
        r = mpx.mpx_irecv_enqueue(buf.data_ptr(), 16, mpx.BYTE, 0, 9, comm[1])
        mpx.mpx_waitall_enqueue([r])
        for _ in range(3):
            mpx.mpx_world_progress(w, raw[2])
        assert _wait_idle(cs[2], 10.0), "a drain pass did not return"
        assert mpx.mpx_stream_pending(ms[1]) > 0
        assert not cs[1].query()
        mpx.mpx_world_abort(w)
        assert _wait_idle(cs[1], 10.0)
        assert mpx.mpx_world_get_error(w) == mpx.ERR_TIMEOUT
        # in drain mode one more pass retires the released operations
        mpx.mpx_world_progress(w, raw[2])
        assert _wait_idle(cs[2], 10.0)
        assert mpx.mpx_stream_pending(ms[1]) == 0
    finally:
        _teardown(mpx, w, raw, ms, comm, cs)
