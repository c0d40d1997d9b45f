"""Serving loop (mpx_serve_run) on the GPU: open-loop requests from many host
threads, admitted by a device-memory budget, through the resident engine.

* every request completes, and the budget was actually contended (requests
  waited for memory) when it is small;
* each sampled item (p2p message or allreduce instance) delivers the same
  bytes in the mix as when it runs alone, and the same as through the plain
  path (an independent implementation: host matching, one copy per message,
  one reduction kernel per allreduce);
* with a caller-supplied schedule (mpx_serve_run_schedule), every delivered
  item and every status equals the CPU oracle's, element by element, in the
  mix (engine and plain path) and alone."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _mpx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_13707_gb300 import mpx
    return mpx


def _cfg(mpx, **kw):
    c = mpx.mpx_serve_config_init()
    c.nthreads = 8
    c.requests = 16000
    c.mean_gap_us = 5.0
    c.min_log2, c.max_log2 = 6, 18
    c.budget_bytes = 64 << 20
    c.sample_every = 97
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _counts(c):
    per = c.requests // c.nthreads
    nar = int(math.floor(c.p_allreduce * per + 0.5))
    msgs = (per - nar) * c.nthreads // 2
    return msgs, nar


def test_serving_mix_alone_and_plain_agree():
    mpx = _mpx()
    c = _cfg(mpx)
    msgs, nar = _counts(c)
    items = msgs + nar
    mix = np.zeros(items, np.uint64)
    src = np.zeros(items, np.uint64)
    res = mpx.mpx_serve_run(c, mix, src)
    assert res["items"] == items and res["completed"] == 2 * msgs + nar * c.nthreads
    sampled = np.nonzero(mix)[0]
    assert len(sampled) >= 5, "too few sampled items"
    # every sampled message arrived as its sender holds it
    p2p = sampled[sampled < msgs]
    assert len(p2p) >= 3
    assert np.array_equal(src[p2p], mix[p2p]), "a delivered payload differs from what was sent"
    # plain path: same schedule, same digests
    plain = np.zeros(items, np.uint64)
    mpx.mpx_serve_run(_cfg(mpx, engine_mode=mpx.ENGINE_PLAIN), plain)
    assert np.array_equal(plain[sampled], mix[sampled]), "plain path delivered different bytes"
    # alone: a few messages and the first sampled allreduce instance
    picks = list(sampled[:3]) + list(sampled[-2:])
    for it in picks:
        alone = np.zeros(items, np.uint64)
        mpx.mpx_serve_run(_cfg(mpx, only_item=int(it), mean_gap_us=0.0), alone)
        assert alone[it] == mix[it], f"item {it}: alone {alone[it]:#x} vs mix {mix[it]:#x}"
    assert any(it >= msgs for it in sampled), "no allreduce instance was sampled"


def test_serving_completes_every_request_under_a_tight_budget():
    mpx = _mpx()
    c = _cfg(mpx, budget_bytes=8 * (1 << 18) * 4, mean_gap_us=0.5, sample_every=0)
    res = mpx.mpx_serve_run(c)
    msgs, nar = _counts(c)
    assert res["completed"] == 2 * msgs + nar * c.nthreads
    assert res["admission_waits"] > 0, "the budget never held a request back"
    assert res["peak_bytes"] <= c.budget_bytes
    assert res["p99_us"] >= res["p50_us"] > 0


# ---------------------------------------------------------------------------
# against the oracle: the same requests as a caller-supplied schedule, every
# delivered item and every status compared element by element
# ---------------------------------------------------------------------------
def _run_schedule(mpx, torch, sched, **cfg_kw):
    dev = torch.device("cuda")
    regions = [torch.from_numpy(r).to(dev) for r in sched["regions"]]
    cap = torch.zeros(int(sched["capture_bytes"]), dtype=torch.uint8, device=dev)
    sts = torch.zeros(int(sched["nstatuses"]) * 24, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    c = _cfg(mpx, nthreads=int(sched["nthreads"]), **cfg_kw)
    res = mpx.mpx_serve_run_schedule(c, sched["calls"], sched["call_lo"], [r.data_ptr() for r in regions],
                                     int(sched["region_bytes"]), cap.data_ptr(), cap.numel(),
                                     sts.data_ptr(), int(sched["nstatuses"]))
    torch.cuda.synchronize()
    from traffic.program import STATUS_DTYPE
    st = np.frombuffer(sts.cpu().numpy().tobytes(), STATUS_DTYPE)
    return res, cap.cpu().numpy(), st


def _item_slices(sched, item):
    """(offset, bytes) of the capture slices an item fills."""
    M = sched["messages"]
    if item < M:
        return [(sched["cap_off"][item], int(sched["mbytes"][item]))]
    e = item - M
    return [(sched["cap_off"][(item, t)], int(sched["abytes"][e])) for t in range(sched["nthreads"])]


@pytest.mark.parametrize("mode", ["engine", "plain"])
def test_serving_schedule_matches_the_oracle(mode):
    """Every p2p payload byte for byte and every status field by field (the
    wildcard-free closed form, P1: the k-th send of a (source, destination,
    tag) pair is the k-th receive), every rank's fixed-order allreduce result
    bit for bit, under a budget small enough that requests wait for memory."""
    mpx = _mpx()
    torch = pytest.importorskip("torch")
    import oracle
    from traffic import gen
    sched = gen.serving_schedule(nthreads=8, requests=4000, max_log2=14)
    p = gen.serving_program(sched)
    ref = oracle.run(p)
    assert ref.error == 0 and not ref.deadlock
    want = ref.buffers[sched["nthreads"]]       # the capture buffer
    # a share of 64 KiB per thread holds the largest epoch's receives (25.6 KB
    # here) but not several epochs': threads that run ahead wait for memory
    kw = {"budget_bytes": 8 * (1 << 16), "mean_gap_us": 0.5}
    if mode == "plain":
        kw["engine_mode"] = mpx.ENGINE_PLAIN
    res, got, st = _run_schedule(mpx, torch, sched, **kw)
    calls = sched["calls"]
    assert res["completed"] == int(np.sum(calls["kind"] != gen.SERVE_WAITALL))
    if mode == "engine":
        assert res["admission_waits"] > 0, "the budget never held a request back"
    assert np.array_equal(got, want), f"{int(np.sum(got != want))} captured bytes differ"
    assert np.array_equal(st, ref.status), "statuses differ"


def test_serving_items_alone_equal_the_mix():
    """An item run alone (its calls only, no pacing) delivers what it delivers
    in the mix, and both equal the oracle: messages and allreduce instances."""
    mpx = _mpx()
    torch = pytest.importorskip("torch")
    import oracle
    from traffic import gen
    full = gen.serving_schedule(nthreads=8, requests=4000, max_log2=14)
    want = oracle.run(gen.serving_program(full)).buffers[full["nthreads"]]
    _, mix, _ = _run_schedule(mpx, torch, full, budget_bytes=8 * (1 << 16), mean_gap_us=2.0)
    M = full["messages"]
    picks = [0, M // 3, M - 1, M, M + full["instances"] - 1]
    for it in picks:
        alone = gen.serving_schedule(nthreads=8, requests=4000, max_log2=14, only_items=[it])
        _, got, _ = _run_schedule(mpx, torch, alone, budget_bytes=8 * (1 << 16), mean_gap_us=0.0)
        for off, n in _item_slices(full, it):
            assert np.array_equal(got[off: off + n], want[off: off + n]), f"item {it} alone vs oracle"
            assert np.array_equal(mix[off: off + n], want[off: off + n]), f"item {it} in the mix vs oracle"
