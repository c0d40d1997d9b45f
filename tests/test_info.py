"""MPI_Info objects and MPIX_Info_set_hex (§3.2), through the C ABI on the host
(no GPU needed), and MPIX_Stream_create from info hints as in Listing 4 (GPU)."""
import struct

import numpy as np
import pytest


@pytest.fixture(scope="module")
def mpx():
    from paper_2208_13707_gb300 import build, mpx as m
    build.build()
    return m


def _code(m, fn):
    try:
        fn()
    except m.MpxError as e:
        return e.code
    return 0


def test_set_get_replace_and_key_order(mpx):
    info = mpx.mpx_info_create()
    try:
        mpx.mpx_info_set(info, "type", "cudaStream_t")
        mpx.mpx_info_set(info, "b", "2")
        mpx.mpx_info_set(info, "a", "1")
        mpx.mpx_info_set(info, "b", "two")          # a second set replaces the value
        assert mpx.mpx_info_get_nkeys(info) == 3
        assert [mpx.mpx_info_get_nthkey(info, k) for k in range(3)] == ["type", "b", "a"]
        assert mpx.mpx_info_get(info, "b") == "two"
        assert mpx.mpx_info_get(info, "missing") is None
        assert mpx.mpx_info_get_valuelen(info, "type") == len("cudaStream_t")
        assert mpx.mpx_info_get(info, "type", buflen=5) == "cuda"  # buflen - 1 characters
    finally:
        mpx.mpx_info_free(info)


def test_hex_encoding_is_the_bytes_in_memory_order(mpx):
    """The stored text is Python's bytes.hex() of the value: two lowercase
    digits per byte, first byte first."""
    info = mpx.mpx_info_create()
    try:
        rng = np.random.default_rng(0x220813707)
        for n in (1, 2, 7, 8, 16, 512):
            v = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
            mpx.mpx_info_set_hex(info, "value", v)
            assert mpx.mpx_info_get(info, "value") == v.hex()
            assert mpx.mpx_info_get_hex(info, "value", n) == v
        # a pointer-sized handle as in Listing 4: little-endian bytes of the integer
        h = 0x00007F12345678A0
        mpx.mpx_info_set_hex(info, "value", struct.pack("<Q", h))
        assert mpx.mpx_info_get(info, "value") == "a0785634127f0000"
        assert struct.unpack("<Q", mpx.mpx_info_get_hex(info, "value", 8))[0] == h
        # upper-case digits written with mpx_info_set read back too
        mpx.mpx_info_set(info, "u", "0A0B")
        assert mpx.mpx_info_get_hex(info, "u", 2) == b"\x0a\x0b"
    finally:
        mpx.mpx_info_free(info)


def test_argument_errors(mpx):
    info = mpx.mpx_info_create()
    try:
        assert _code(mpx, lambda: mpx.mpx_info_set(info, "", "x")) == mpx.ERR_ARG
        assert _code(mpx, lambda: mpx.mpx_info_set(info, "k" * 256, "x")) == mpx.ERR_ARG
        mpx.mpx_info_set(info, "k" * 255, "x")                     # the longest key
        assert _code(mpx, lambda: mpx.mpx_info_set(info, "v", "x" * 1025)) == mpx.ERR_ARG
        mpx.mpx_info_set(info, "v", "x" * 1024)                     # the longest value
        assert _code(mpx, lambda: mpx.mpx_info_set_hex(info, "h", b"\0" * 513)) == mpx.ERR_ARG
        mpx.mpx_info_set(info, "h", "0g")
        assert _code(mpx, lambda: mpx.mpx_info_get_hex(info, "h", 1)) == mpx.ERR_ARG   # not hex
        assert _code(mpx, lambda: mpx.mpx_info_get_hex(info, "v", 8)) == mpx.ERR_ARG   # wrong length
        assert mpx.mpx_info_get_hex(info, "absent", 8) is None
        assert _code(mpx, lambda: mpx.mpx_info_get_nthkey(info, 3)) == mpx.ERR_ARG
    finally:
        mpx.mpx_info_free(info)


@pytest.mark.gpu
def test_stream_from_info_hints_listing4_pattern(mpx):
    """Listing 4: the CUDA stream goes into an info object as type
    "cudaStream_t" plus its hex-encoded handle; the MPIX stream created from it
    enqueues on that CUDA stream.  MPI_INFO_NULL gives a library-owned one."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    cfg = mpx.mpx_world_config_init()
    cfg.max_streams = 4
    w = mpx.mpx_world_create(2, cfg)
    cs = mpx.mpx_cuda_stream_create()
    info = mpx.mpx_info_create()
    made = []
    try:
        mpx.mpx_info_set(info, "type", "cudaStream_t")
        mpx.mpx_info_set_hex(info, "value", struct.pack("<Q", cs))
        s0 = mpx.mpx_stream_create_info(w, 0, info)
        made.append(s0)
        assert mpx.mpx_stream_get_cuda_stream(s0) == cs
        s1 = mpx.mpx_stream_create_info(w, 1, None)               # MPI_INFO_NULL
        made.append(s1)
        own = mpx.mpx_stream_get_cuda_stream(s1)
        assert own not in (0, cs)
        # hints the call rejects
        bad = mpx.mpx_info_create()
        try:
            mpx.mpx_info_set(bad, "type", "hipStream_t")
            mpx.mpx_info_set_hex(bad, "value", struct.pack("<Q", cs))
            assert _code(mpx, lambda: mpx.mpx_stream_create_info(w, 0, bad)) == mpx.ERR_ARG
            mpx.mpx_info_set(bad, "type", "cudaStream_t")
            mpx.mpx_info_set(bad, "mpx_exclusive", "maybe")
            assert _code(mpx, lambda: mpx.mpx_stream_create_info(w, 0, bad)) == mpx.ERR_ARG
        finally:
            mpx.mpx_info_free(bad)
        comm = mpx.mpx_stream_comm_create(w, [s0, s1])
        src = torch.arange(256, dtype=torch.int32, device="cuda")
        dst = torch.zeros(256, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        mpx.mpx_send_enqueue(src.data_ptr(), 256, mpx.INT32, 1, 3, comm[0])
        mpx.mpx_recv_enqueue(dst.data_ptr(), 256, mpx.INT32, 0, 3, comm[1], 0)
        torch.cuda.ExternalStream(own).synchronize()
        torch.cuda.ExternalStream(cs).synchronize()
        assert torch.equal(dst, src)
        for h in comm:
            mpx.mpx_comm_free(h)
    finally:
        mpx.mpx_info_free(info)
        mpx.mpx_world_stop(w, 10000)
        import time
        for s_ in made:
            for _ in range(2000):
                try:
                    mpx.mpx_stream_free(s_)
                    break
                except mpx.MpxError as e:
                    if e.code != mpx.ERR_PENDING:
                        raise
                    time.sleep(5e-4)
        mpx.mpx_world_free(w)
        mpx.mpx_cuda_stream_destroy(cs)
