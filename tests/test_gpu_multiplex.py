"""GPU parity for multiplex stream communicators (§3.5): the CUDA path through
the C ABI against the CPU oracle, plus the host-side argument checks."""
import numpy as np
import pytest

import oracle
from traffic import gen
from traffic.program import ISEND, SEND

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
    out = gpu.run(p, mode=mode, timeout_s=45)
    assert out.finished, "GPU run did not finish before the deadline"
    assert out.world_error == 0
    for k, (a, b) in enumerate(zip(out.buffers, ref.buffers)):
        if not np.array_equal(a, b):
            diff = np.nonzero(a != b)[0]
            raise AssertionError(f"buffer {k}: {len(diff)} bytes differ, first at {diff[:8]}")
    if p.nstatus:
        assert np.array_equal(out.status, ref.status), "statuses differ"
    return out, ref


def _wildcard_program(k):
    """The k-th seeded random multiplex program that completes (programs whose
    wildcards strand a receive deadlock by construction and are passed over)."""
    seed, found = 0, -1
    while True:
        counts = ((2, 3), (3, 1), (1, 4), (2, 2))[seed % 4]
        p = gen.multiplex_small(gen.SEED_BASE + 900 + seed, nranks=2, counts=counts, nmsg=8)
        if not oracle.run(p).deadlock:
            found += 1
            if found == k:
                return p
        seed += 1


@pytest.mark.parametrize("k", range(16))
def test_multiplex_wildcards_drain_exact(k):
    """Every operation is visible before the first pass, so the engine's
    outcome is the oracle's, wildcards (ANY_SOURCE, ANY_INDEX, ANY_TAG)
    included."""
    _gpu()
    _compare(_wildcard_program(k), "drain")


@pytest.mark.parametrize("mode", ["persistent", "drain"])
def test_multiplex_wildcard_free_three_ranks(mode):
    """Without wildcards the outcome is unique: a resident engine must give it too."""
    p = gen.multiplex_small(gen.SEED_BASE + 950, nranks=3, counts=(2, 1, 3), nmsg=40,
                            p_any_src=0.0, p_any_idx=0.0, p_any_tag=0.0, p_blocking=0.2,
                            p_wait=0.0, max_count=64)
    _compare(p, mode)


def test_n_to_one_drain_exact():
    _compare(gen.n_to_one(nranks=4, threads=4, msgs=8, max_bytes=4096), "drain")


def test_n_to_one_resident_engine_is_legal():
    """Live traffic into one (ANY_SOURCE, ANY_INDEX, ANY_TAG) poller: every
    message arrives once, each sender's messages in order, with the sender's
    rank, index, tag and bytes in the status and its payload in the buffer."""
    gpu = _gpu()
    nranks, threads, msgs = 4, 4, 16
    p = gen.n_to_one(nranks=nranks, threads=threads, msgs=msgs, max_bytes=8192)
    out = gpu.run(p, mode="persistent", timeout_s=45)
    assert out.finished and out.world_error == 0
    st = out.status
    assert np.all(st["error"] == 0)
    # the send of (rank r, index i) with tag k
    sends = {}
    for j in np.nonzero(np.isin(p.ops["kind"], [SEND, ISEND]))[0]:
        o = p.ops[j]
        r, i = p.member(int(o["comm"]), int(o["stream"]))
        sends[(r, i, int(o["tag"]))] = o
    order = {}
    recvs = [j for j in np.nonzero(p.ops["kind"] == 3)[0]]
    init = p.fresh_buffers()
    for q, j in enumerate(recvs):
        key = (int(st["source"][q]), int(st["source_index"][q]), int(st["tag"][q]))
        assert key in sends, key
        order.setdefault(key[:2], []).append(key[2])
        so, ro = sends[key], p.ops[j]
        n = 4 * int(so["count"])
        assert int(st["bytes"][q]) == n
        data = init[int(so["buf"])][int(so["off"]): int(so["off"]) + n]
        got = out.buffers[int(ro["buf"])][int(ro["off"]): int(ro["off"]) + n]
        assert np.array_equal(got, data), key
    senders = [(r, i) for r in range(nranks) for i in range(threads) if (r, i) != (0, 0)]
    assert sorted(order) == senders
    for s in senders:
        assert order[s] == list(range(msgs)), (s, order[s])


def test_multiplex_argument_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_13707_gb300 import mpx
    cfg = mpx.mpx_world_config_init()
    cfg.max_streams = 8
    cfg.max_comms = 4
    w = mpx.mpx_world_create(2, cfg)
    raw = [mpx.mpx_cuda_stream_create() for _ in range(5)]
    st = [mpx.mpx_stream_create(w, r, raw[k], mpx.STREAM_DEFAULT)
          for k, r in enumerate((0, 0, 1, 1, 1))]
    comms = []

    def code(fn):
        try:
            fn()
        except mpx.MpxError as e:
            return e.code
        return 0

    try:
        # a rank with no stream, a stream of another rank, a stream twice
        assert code(lambda: mpx.mpx_stream_comm_create_multiple(w, [[], [st[2]]])) == mpx.ERR_ARG
        assert code(lambda: mpx.mpx_stream_comm_create_multiple(w, [[st[2]], [st[3]]])) == mpx.ERR_ARG
        assert code(lambda: mpx.mpx_stream_comm_create_multiple(w, [[st[0], st[0]], [st[2]]])) == mpx.ERR_ARG
        mux = mpx.mpx_stream_comm_create_multiple(w, [[st[0], st[1]], [st[2], st[3], st[4]]])
        comms.append(mux)
        plain = mpx.mpx_stream_comm_create(w, [st[0], st[2]])
        comms.append(plain)
        # 5 members of 2 ranks take 3 slots, the plain comm 1: the world's 4 are used
        assert code(lambda: mpx.mpx_stream_comm_create(w, [st[1], st[3]])) == mpx.ERR_NO_MEM
        buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
        p = buf.data_ptr()
        # plain calls and collectives on a multiplex handle, multiplex calls on a plain one
        assert code(lambda: mpx.mpx_isend_enqueue(p, 4, mpx.BYTE, 1, 0, mux[0])) == mpx.ERR_COMM
        assert code(lambda: mpx.mpx_allreduce_enqueue(p, p, 4, mpx.BYTE, mpx.SUM, mux[0])) == mpx.ERR_COMM
        assert code(lambda: mpx.mpx_barrier_enqueue(mux[0])) == mpx.ERR_COMM
        assert code(lambda: mpx.mpx_stream_isend_enqueue(p, 4, mpx.BYTE, 1, 0, plain[0], 0, 0)) == mpx.ERR_COMM
        # indices out of range
        assert code(lambda: mpx.mpx_stream_isend_enqueue(p, 4, mpx.BYTE, 1, 0, mux[0], 2, 0)) == mpx.ERR_ARG
        assert code(lambda: mpx.mpx_stream_isend_enqueue(p, 4, mpx.BYTE, 1, 0, mux[0], 0, 3)) == mpx.ERR_ARG
        assert code(lambda: mpx.mpx_stream_irecv_enqueue(p, 4, mpx.BYTE, 0, 0, mux[1], 2, 0)) == mpx.ERR_ARG
        assert code(lambda: mpx.mpx_stream_irecv_enqueue(p, 4, mpx.BYTE, mpx.ANY_SOURCE, 0, mux[1], 3, 0)) == mpx.ERR_ARG
        assert code(lambda: mpx.mpx_stream_irecv_enqueue(p, 4, mpx.BYTE, 0, 0, mux[1], 0, 3)) == mpx.ERR_ARG
        assert code(lambda: mpx.mpx_stream_isend_enqueue(p, 4, mpx.BYTE, 2, 0, mux[0], 0, 0)) == mpx.ERR_RANK
        assert code(lambda: mpx.mpx_stream_isend_enqueue(p, 4, mpx.BYTE, 1, -3, mux[0], 0, 0)) == mpx.ERR_TAG
        # a matched pair across the two ranks' second streams, status with the index
        stat = torch.zeros(24, dtype=torch.uint8, device="cuda")
        src = torch.arange(16, dtype=torch.uint8, device="cuda")
        dst = torch.zeros(16, dtype=torch.uint8, device="cuda")
        r1 = mpx.mpx_stream_isend_enqueue(src.data_ptr(), 16, mpx.BYTE, 1, 7, mux[0], 1, 2)
        r2 = mpx.mpx_stream_irecv_enqueue(dst.data_ptr(), 16, mpx.BYTE, 0, mpx.ANY_TAG, mux[1],
                                          mpx.ANY_INDEX, 2)
        mpx.mpx_wait_enqueue(r1, 0)
        mpx.mpx_wait_enqueue(r2, stat.data_ptr())
        torch.cuda.synchronize()
        for h in raw:
            torch.cuda.ExternalStream(h).synchronize()
        assert torch.equal(dst, src)
        s = np.frombuffer(stat.cpu().numpy().tobytes(), np.int32)
        assert s[:4].tolist() == [0, 7, 0, 1] and int(stat.cpu().numpy().view(np.int64)[2]) == 16
    finally:
        for cl in comms:
            for h in cl:
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
