"""The benchmark's multi-GPU form is replicas (one independent world per
rank, no collective on the data path).  Its whole-job aggregation — the
slowest rank's time, the units of every rank — is checked here with two
gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) seconds for 100 * (r + 1) units
        secs, value = bench.whole_job(float(rank + 1), 100 * (rank + 1), dist, "cpu")
        out[rank] = (secs, value)
    finally:
        dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank_and_all_units():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        secs, value = out[r]
        assert secs == pytest.approx(2.0)
        assert value == pytest.approx((100 + 200) / 2.0)


def test_whole_job_single_process():
    sys.path.insert(0, ROOT)
    import bench
    secs, value = bench.whole_job(0.5, 40)
    assert secs == 0.5 and value == pytest.approx(80.0)
