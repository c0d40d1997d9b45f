"""Host-thread 8-byte message rate under the three locking disciplines of the
multithreaded-rate experiment (§5.3, Fig. 3): every message arrives, in order,
whatever the discipline, thread count or window; arguments are checked."""
import pytest


@pytest.fixture(scope="module")
def mpx():
    from paper_2208_13707_gb300 import build, mpx as m
    build.build()
    return m


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("threads,window", [(1, 1), (2, 7), (3, 64), (2, 1024)])
def test_every_message_arrives_in_order(mpx, mode, threads, window):
    # more messages than a channel's 1024-entry queue, and a ragged last window
    r = mpx.mpx_hostrate_run(threads, mode, messages=5000 + 13, window=window)
    assert r["errors"] == 0
    assert r["msgs_per_s"] > 0 and r["seconds"] > 0


def test_argument_checks(mpx):
    for args in [(0, 2), (513, 2), (1, 3)]:
        with pytest.raises(mpx.MpxError) as e:
            mpx.mpx_hostrate_run(*args, messages=10)
        assert e.value.code == mpx.ERR_ARG
    for kw in [dict(messages=0), dict(window=0), dict(window=1025)]:
        with pytest.raises(mpx.MpxError):
            mpx.mpx_hostrate_run(1, 2, **kw)
