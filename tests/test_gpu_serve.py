"""Serving loop (mpx_serve_run) on the GPU: open-loop requests from many host
threads, admitted by a device-memory budget, through the resident engine.

* every request completes, and the budget was actually contended (requests
  waited for memory) when it is small;
* each sampled item (p2p message or allreduce instance) delivers the same
  bytes in the mix as when it runs alone, and the same as through the plain
  path (an independent implementation: host matching, one copy per message,
  one reduction kernel per allreduce)."""
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
