"""The test-side checkers, pinned on the CPU: reading a run's matching back
from its delivered payloads must reproduce a known match map."""
import numpy as np

import oracle
from traffic import gen

from checks import infer_match_from_payloads, validity_violations


def _unmatched(prog):
    o = oracle.run(prog)
    if not o.deadlock:
        return None
    k = prog.ops["kind"]
    return [j for j in range(len(prog.ops)) if k[j] in (1, 3) and o.match[j] < 0]


def test_payload_inference_recovers_the_match_map():
    """Non-laminar wildcards ((ANY_SOURCE, exact tag) receives) with
    truncations: the map inferred from the oracle's buffers and statuses is
    the oracle's own map, and it passes the validity checker."""
    p = gen.batching(nranks=16, streams_per_rank=2, nmsg=3000, max_bytes=16 << 10,
                     seed=gen.SEED_BASE + 2 + 7000, fixup=_unmatched)
    o = oracle.run(p)
    assert not o.deadlock and o.error == 0
    assert np.any(p.ops["peer"] == -2)          # ANY_SOURCE receives are present
    m, problems = infer_match_from_payloads(p, o.buffers, o.status)
    assert problems == []
    assert np.array_equal(m, o.match)
    assert validity_violations(p, m, require_complete=True) == []


def test_payload_inference_reports_a_wrong_delivery():
    """A receive buffer whose bytes no send explains is reported."""
    p = gen.batching(nranks=8, streams_per_rank=1, nmsg=200, max_bytes=4096,
                     seed=gen.SEED_BASE + 2 + 7001, laminar=True)
    o = oracle.run(p)
    bufs = [b.copy() for b in o.buffers]
    r = int(np.nonzero(p.ops["kind"] == 3)[0][0])
    ro = p.ops[r]
    bufs[int(ro["buf"])][int(ro["off"])] ^= 0xFF
    _, problems = infer_match_from_payloads(p, bufs, o.status)
    assert any(f"recv {r}:" in s for s in problems)
