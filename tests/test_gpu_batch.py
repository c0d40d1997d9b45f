"""Batch submission (mpx_enqueue_batch) on the GPU against the oracle: the
batching workload's shape (64 ranks x 4 MPIX streams, four stream comms,
uniform sources, destinations and tags, log-uniform 8 B - 64 KB messages of
mixed dtypes, ANY_TAG and ANY_SOURCE receives) at a size the oracle finishes
in seconds, through the persistent engine, drain passes and the plain path.
Large rounds match from domain-sorted post lists, so these cases cover that
path; the other parity tests' small rounds cover the scanning one."""
import numpy as np
import pytest

import oracle
from traffic import gen
from traffic.program import ERR_TRUNCATE

from checks import infer_match_from_payloads, validity_violations

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from traffic import gpu
    return gpu


def _program(nmsg=8000, seed_off=0, nranks=64, streams_per_rank=4):
    return gen.batching(nranks=nranks, streams_per_rank=streams_per_rank, nmsg=nmsg,
                        max_bytes=64 << 10, laminar=True, seed=gen.SEED_BASE + 2 + 1000 * seed_off)


def _check(r, ref):
    bufs, status = r.results()
    serr, werr = r.errors()
    assert werr == 0 and not any(serr), (werr, serr)
    for k, (a, b) in enumerate(zip(bufs, ref.buffers)):
        if not np.array_equal(a, b):
            diff = np.nonzero(a != b)[0]
            raise AssertionError(f"buffer {k}: {len(diff)} bytes differ, first at {diff[:8]}")
    assert np.array_equal(status, ref.status), "statuses differ"


# Drain passes run on a stream of their own; with every one of 256 streams
# stopped at its waitall, each of CUDA's hardware queues can hold a blocked
# wait in front of the pass.  The drain case therefore uses 16 ranks x 1
# stream (fewer streams than queues); the persistent engine is resident
# before any wait is enqueued and has no such limit.
@pytest.mark.parametrize("mode,exclusive,shape", [("persistent", True, (64, 4)),
                                                  ("persistent", False, (64, 4)),
                                                  ("drain", True, (16, 1)),
                                                  ("drain", False, (16, 1)),
                                                  ("graph", True, (64, 4)),
                                                  ("plain", True, (64, 4))])
def test_batched_small_messages_match_the_oracle(mode, exclusive, shape):
    gpu = _gpu()
    p = _program(nranks=shape[0], streams_per_rank=shape[1])
    ref = oracle.run(p)
    assert ref.error == 0 and not ref.deadlock
    r = gpu.BatchRunner(p, mode=mode, exclusive=exclusive, timeout_s=60)
    try:
        assert r.step(), "step did not finish"
        _check(r, ref)
        # a second step over the same buffers gives the same bytes and statuses
        assert r.step(), "second step did not finish"
        _check(r, ref)
    finally:
        r.close()


def test_batched_steps_after_buffer_reset_persistent():
    gpu = _gpu()
    p = _program(nmsg=20000, seed_off=1)
    ref = oracle.run(p)
    r = gpu.BatchRunner(p, mode="persistent", timeout_s=60)
    try:
        for _ in range(3):
            r.reset_buffers()
            assert r.step()
            _check(r, ref)
    finally:
        r.close()


def test_recorded_step_replays_and_returns_streams_to_host_enqueue():
    """A recorded step (CUDA graph) replayed five times gives the oracle's
    bytes and statuses; after mpx_step_free the same streams take host
    enqueue calls again (their sequence numbers continued on the device)."""
    gpu = _gpu()
    from paper_2208_13707_gb300 import mpx
    p = _program(nmsg=4000, seed_off=2, nranks=8, streams_per_rank=2)
    ref = oracle.run(p)
    r = gpu.BatchRunner(p, mode="graph", timeout_s=60)
    try:
        for _ in range(5):
            r.enqueue()
        assert r.finish()
        assert mpx.mpx_step_get_error(r.step_handle) == 0
        _check(r, ref)
        # host enqueue on a stream owned by the step is refused
        with pytest.raises(mpx.MpxError) as e:
            mpx.mpx_enqueue_batch(r.ops[:1])
        assert e.value.code == mpx.ERR_STATE
        mpx.mpx_step_free(r.step_handle)
        r.graph = False
        r.reset_buffers()
        assert r.step(), "host-enqueued step after the recorded ones did not finish"
        _check(r, ref)
    finally:
        r.close()


def test_per_cta_mover_schedule_matches_the_oracle():
    """Movers that each own a queue of tasks (MPX_MOVERS_PER_CTA) deliver the
    same bytes and statuses as the shared work list."""
    gpu = _gpu()
    p = _program(nmsg=8000, seed_off=3)
    ref = oracle.run(p)
    r = gpu.BatchRunner(p, mode="persistent", cfg_over={"mover_schedule": 1}, timeout_s=60)
    try:
        assert r.step()
        _check(r, ref)
    finally:
        r.close()


# ---------------------------------------------------------------------------
# non-laminar wildcards: (ANY_SOURCE, exact tag) receives next to (s, ANY_TAG)
# ones, widened to (ANY_SOURCE, ANY_TAG) only where the oracle finds a
# receive that can never match; some exact receives truncate
# ---------------------------------------------------------------------------
def _unmatched(prog):
    o = oracle.run(prog)
    if not o.deadlock:
        return None
    k = prog.ops["kind"]
    return [j for j in range(len(prog.ops)) if k[j] in (1, 3) and o.match[j] < 0]


def _nonlaminar(nranks=64, streams_per_rank=4, nmsg=8000, seed_off=7):
    p = gen.batching(nranks=nranks, streams_per_rank=streams_per_rank, nmsg=nmsg,
                     max_bytes=64 << 10, seed=gen.SEED_BASE + 2 + 1000 * seed_off, fixup=_unmatched)
    ref = oracle.run(p)
    assert ref.error == 0 and not ref.deadlock
    assert np.any(p.ops["peer"] == -2) and np.any(ref.status["error"] == ERR_TRUNCATE)
    return p, ref


def test_nonlaminar_wildcards_recorded_step_exact():
    """The recorded step publishes every descriptor before its engine pass, so
    the canonical round order holds and the outcome equals the oracle's, byte
    for byte and status for status, on two replays."""
    gpu = _gpu()
    p, ref = _nonlaminar()
    r = gpu.BatchRunner(p, mode="graph", timeout_s=60)
    try:
        for _ in range(2):
            r.enqueue()
            assert r.finish(), "step did not finish"
            bufs, status = r.results()
            for k, (a, b) in enumerate(zip(bufs, ref.buffers)):
                assert np.array_equal(a, b), f"buffer {k} differs"
            assert np.array_equal(status, ref.status), "statuses differ"
            serr, werr = r.errors()
            assert werr == ERR_TRUNCATE
    finally:
        r.close()


def test_nonlaminar_wildcards_persistent_engine_is_legal():
    """Live traffic into a resident engine: descriptors of different streams
    arrive at different ticks, so an ANY_SOURCE receive may legally take
    another sender's message than in the canonical order.  The matching read
    back from the delivered bytes must be an MPI-legal outcome (every receive
    matched once, compatible, no overtaking), with statuses and truncation
    errors that fit the sends it names."""
    gpu = _gpu()
    p, ref = _nonlaminar(seed_off=8)
    r = gpu.BatchRunner(p, mode="persistent", timeout_s=60)
    try:
        assert r.step(), "step did not finish"
        bufs, status = r.results()
    finally:
        r.close()
    match, problems = infer_match_from_payloads(p, bufs, status)
    assert problems == [], problems[:5]
    assert validity_violations(p, match, require_complete=True) == []
