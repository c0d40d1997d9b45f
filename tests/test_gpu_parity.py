"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, byte
for byte on payloads and field by field on statuses."""
import numpy as np
import pytest

import oracle
from traffic import gen
from traffic.program import (ANY_SOURCE, ANY_TAG, ERR_TRUNCATE, MODE_FIXED, MODE_TREE, T_BYTE,
                             T_DOUBLE, T_FLOAT, T_INT32, T_INT64, ProgramBuilder)

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from traffic import gpu
    return gpu


def _compare(p, mode="persistent", exclusive=False, status=True, cfg_over=None, timeout_s=45,
             world_error=None):
    gpu = _gpu()
    ref = oracle.run(p)
    assert ref.error == 0, "oracle rejected the program"
    assert not ref.deadlock
    if world_error is None:  # the first asynchronous error the oracle's statuses imply
        world_error = ERR_TRUNCATE if p.nstatus and np.any(ref.status["error"] == ERR_TRUNCATE) else 0
    out = gpu.run(p, mode=mode, exclusive=exclusive, cfg_over=cfg_over, timeout_s=timeout_s)
    assert out.finished, "GPU run did not finish before the deadline"
    assert out.world_error == world_error, f"world error {out.world_error}"
    for k, (a, b) in enumerate(zip(out.buffers, ref.buffers)):
        if not np.array_equal(a, b):
            diff = np.nonzero(a != b)[0]
            raise AssertionError(f"buffer {k}: {len(diff)} bytes differ, first at {diff[:8]}")
    if status and p.nstatus:
        assert np.array_equal(out.status, ref.status), "statuses differ"
    return out, ref


def test_listing4_gives_four():
    p = gen.listing4(1 << 20)
    out, _ = _compare(p)
    assert np.all(out.buffers[p.meta["dy"]].view(np.float32) == 4.0)


def test_listing3_four_stream_comms():
    _compare(gen.listing3(4, 100))


@pytest.mark.parametrize("exclusive", [False, True])
def test_tiny_pairs_blocking_sends_and_permuted_recvs(exclusive):
    _compare(gen.tiny_pairs(nmsg=1000), exclusive=exclusive)


@pytest.mark.parametrize("mode", ["persistent", "drain"])
def test_ring_exchange_small(mode):
    p = gen.ring_exchange(nranks=8, n=1 << 12, steps=4, min_bytes=256, max_bytes=256 << 10)
    _compare(p, mode=mode)


def test_resident_engine_leaves_room_for_compute_kernels():
    """A resident engine asked for 512 threads per CTA would take every
    register of every SM (128 per thread), and the axpy each rank runs before
    its sends could never start.  The world caps a resident engine's threads
    so that half the registers stay free; the ring steps then finish (a
    short watchdog turns a regression into a world error, not a hang)."""
    p = gen.ring_exchange(nranks=8, n=1 << 12, steps=2, min_bytes=256, max_bytes=64 << 10)
    _compare(p, mode="persistent", cfg_over={"engine_threads": 512, "watchdog_ns": 3_000_000_000})


def _device_rings_or_skip():
    from paper_2208_13707_gb300 import mpx
    cfg = mpx.mpx_world_config_init()
    cfg.ring_placement = mpx.RINGS_DEVICE
    cfg.max_streams = 2
    try:
        w = mpx.mpx_world_create(1, cfg)
    except mpx.MpxError as e:
        if e.code == mpx.ERR_UNSUPPORTED:
            pytest.skip("no direct host access to managed device memory")
        raise
    mpx.mpx_world_free(w)


@pytest.mark.parametrize("mode", ["persistent", "drain"])
def test_ring_exchange_with_rings_in_device_memory(mode):
    """Submission rings, waitall lists and stream control lines in device
    memory written by the host through the coherent link: same outcome."""
    _gpu()
    _device_rings_or_skip()
    from paper_2208_13707_gb300 import mpx
    p = gen.ring_exchange(nranks=8, n=1 << 12, steps=4, min_bytes=256, max_bytes=256 << 10)
    _compare(p, mode=mode, cfg_over={"ring_placement": mpx.RINGS_DEVICE})


def test_batching_with_rings_in_device_memory():
    _gpu()
    _device_rings_or_skip()
    from paper_2208_13707_gb300 import mpx
    p = gen.batching(nranks=8, streams_per_rank=2, nmsg=2000, max_bytes=4096, laminar=True,
                     seed=gen.SEED_BASE + 11)
    _compare(p, mode="persistent", cfg_over={"ring_placement": mpx.RINGS_DEVICE})


@pytest.mark.parametrize("schedule", [1])
def test_ring_exchange_per_cta_movers(schedule):
    """Multi-tile messages and vector layouts with each mover owning its tasks."""
    p = gen.ring_exchange(nranks=4, n=1 << 16, steps=3, min_bytes=100_000, max_bytes=3 << 20)
    _compare(p, mode="drain", cfg_over={"mover_schedule": schedule, "tile_bytes": 16 << 10})


def test_ring_exchange_tiles_and_ragged_tail():
    # messages up to 3 MB: many tiles per message, TMA bulk and strided paths
    p = gen.ring_exchange(nranks=4, n=1 << 16, steps=3, min_bytes=100_000, max_bytes=3 << 20)
    _compare(p, cfg_over={"tile_bytes": 65536})


@pytest.mark.parametrize("mode", [MODE_FIXED, MODE_TREE])
def test_allreduce_matches_oracle(mode):
    dts = (T_INT64, T_FLOAT, T_INT32, T_BYTE, T_DOUBLE) if mode == MODE_FIXED else (T_FLOAT,)
    p = gen.allreduce_suite(nranks=16, sizes=(1, 7, 1024, 65537), dtypes=dts, modes=(mode,))
    gpu = _gpu()
    ref = oracle.run(p)
    out = gpu.run(p, timeout_s=45)
    assert out.finished and out.world_error == 0
    for inst in p.meta["instances"]:
        for r in range(p.nranks):
            b = inst["recv"][r]
            if mode == MODE_FIXED:
                assert np.array_equal(out.buffers[b], ref.buffers[b])
            else:
                xs = [p.buf_init[inst["send"][k]].view(np.float32) for k in range(p.nranks)]
                s64, a64 = oracle.sum_f32_ref(xs)
                y = out.buffers[b].view(np.float32).astype(np.float64)
                assert np.all(np.abs(y - s64) <= 1e-6 * a64 + 1e-30)


def test_allreduce_in_place_tree():
    p = gen.allreduce_suite(nranks=16, sizes=(4099,), dtypes=(T_FLOAT,), modes=(MODE_TREE,), in_place=True)
    gpu = _gpu()
    out = gpu.run(p, timeout_s=45)
    assert out.finished and out.world_error == 0
    inst = p.meta["instances"][0]
    xs = [p.buf_init[inst["recv"][k]].view(np.float32) for k in range(p.nranks)]
    s64, a64 = oracle.sum_f32_ref(xs)
    for r in range(p.nranks):
        y = out.buffers[inst["recv"][r]].view(np.float32).astype(np.float64)
        assert np.all(np.abs(y - s64) <= 1e-6 * a64 + 1e-30)


def _completing_random_small(i, **kw):
    """Case i of the random wildcard programs: seed i, or, when the oracle finds
    that program deadlocks by construction (blocking calls in a cycle), the
    first of the derived seeds 1000 * (i + 1) + k, k = 1, 2, ... that completes."""
    k = 0
    while True:
        seed = i if k == 0 else 1000 * (i + 1) + k
        p = gen.random_small(seed, **kw)
        if not oracle.run(p).deadlock:
            return p
        k += 1
        assert k < 200, "no completing program among the derived seeds"


@pytest.mark.parametrize("case", range(24))
def test_random_wildcard_programs_drain_exact(case):
    _compare(_completing_random_small(case, nranks=3, nmsg=6), mode="drain")


def test_halo_exchange_small():
    _compare(gen.halo3d(sub=16, steps=2))


def _unmatched_receives(prog):
    """Receives the oracle leaves unmatched (their wildcards get widened)."""
    o = oracle.run(prog)
    if not o.deadlock:
        return None
    k = prog.ops["kind"]
    return [j for j in range(len(prog.ops)) if k[j] in (1, 3) and o.match[j] < 0]


def test_batching_wildcards_drain_exact():
    p = gen.batching(nranks=8, streams_per_rank=2, nmsg=3000, max_bytes=64 << 10,
                     fixup=_unmatched_receives)
    _compare(p, mode="drain")


def test_truncation_and_any_tag_status():
    b = ProgramBuilder(2)
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    src = b.buffer(np.arange(1, 161, dtype=np.uint8))
    dst = b.buffer(np.full(256, 0xEE, np.uint8))
    st = b.status_slots(2)
    b.send(g0, c, src, 0, 40, T_INT32, 1, 5)
    b.send(g0, c, src, 0, 3, T_INT32, 1, 9)
    b.recv(g1, c, dst, 4, 6, T_INT32, 0, 5, st)
    b.recv(g1, c, dst, 64, 10, T_INT32, ANY_SOURCE, ANY_TAG, st + 1)
    p = b.build()
    out, ref = _compare(p, world_error=ERR_TRUNCATE)   # truncation is a sticky async error
    assert out.status[0]["error"] == ERR_TRUNCATE and out.status[1]["tag"] == 9


def test_zero_count_messages():
    b = ProgramBuilder(2)
    g0, g1 = b.stream(0), b.stream(1)
    c = b.comm([g0, g1])
    x = b.buffer(64)
    st = b.status_slots(1)
    b.send(g0, c, x, 0, 0, T_FLOAT, 1, 1)
    b.recv(g1, c, x, 0, 0, T_FLOAT, 0, 1, st)
    h = b.isend(g1, c, x, 0, 0, T_BYTE, 0, 2)
    b.wait(g1, h)
    b.recv(g0, c, x, 32, 4, T_BYTE, 1, 2)
    _compare(b.build())


# ---------------------------------------------------------------------------
# the plain path (host matching, one copy per operation) on wildcard-free
# traffic, where the outcome is unique
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["tiny", "ring", "halo", "allreduce"])
def test_plain_path_matches_oracle(name):
    p = {"tiny": lambda: gen.tiny_pairs(nmsg=300),
         "ring": lambda: gen.ring_exchange(nranks=8, n=1 << 12, steps=3, min_bytes=256, max_bytes=256 << 10),
         "halo": lambda: gen.halo3d(sub=16, steps=2),
         "allreduce": lambda: gen.allreduce_suite(nranks=8, sizes=(1, 1000), dtypes=(T_INT64, T_FLOAT),
                                                  modes=(MODE_FIXED,))}[name]()
    _compare(p, mode="plain")


def test_enqueue_rejects_counts_whose_bytes_overflow():
    """Counts whose byte span exceeds 2^60 are refused with MPX_ERR_ARG before
    anything is published (p2p calls, collectives, the plain path)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_13707_gb300 import mpx
    for mode in (mpx.ENGINE_DRAIN, mpx.ENGINE_PLAIN):
        cfg = mpx.mpx_world_config_init()
        cfg.engine_mode = mode
        cfg.max_streams = 4
        w = mpx.mpx_world_create(2, cfg)
        raw = [mpx.mpx_cuda_stream_create() for _ in range(2)]
        ms = [mpx.mpx_stream_create(w, r, raw[r]) for r in range(2)]
        comm = mpx.mpx_stream_comm_create(w, ms)
        vec = mpx.mpx_type_vector(1 << 16, 1, 1 << 20, mpx.DOUBLE)   # 2^39-byte extent
        try:
            calls = [lambda: mpx.mpx_isend_enqueue(64, 1 << 62, mpx.DOUBLE, 1, 0, comm[0]),
                     lambda: mpx.mpx_irecv_enqueue(64, 1 << 40, vec, 0, 0, comm[1]),
                     lambda: mpx.mpx_send_enqueue(64, -1, mpx.BYTE, 1, 0, comm[0])]
            if mode == mpx.ENGINE_DRAIN:
                calls += [lambda: mpx.mpx_allreduce_enqueue(64, 128, 1 << 60, mpx.INT64, mpx.SUM, comm[0]),
                          lambda: mpx.mpx_allgather_enqueue(64, 128, 1 << 58, mpx.BYTE, comm[0]),
                          lambda: mpx.mpx_bcast_enqueue(64, 1 << 61, mpx.BYTE, 0, comm[0])]
            for call in calls:
                with pytest.raises(mpx.MpxError) as e:
                    call()
                assert e.value.code == mpx.ERR_ARG
            assert all(mpx.mpx_stream_pending(s) == 0 for s in ms)
        finally:
            mpx.mpx_type_free(vec)
            for c in comm:
                mpx.mpx_comm_free(c)
            for s in ms:
                mpx.mpx_stream_free(s)
            mpx.mpx_world_free(w)
            for h in raw:
                mpx.mpx_cuda_stream_destroy(h)
