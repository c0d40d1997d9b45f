"""Autotuner for the engine's copy schedule (tile size, the size from which
contiguous tiles move by TMA bulk copy, engine CTAs, threads per CTA, and
whether movers share one work list of tiles or each owns a queue of tasks).

`autotune(sizes)` times each candidate world configuration on a synthetic
sample of the caller's message mix: R ranks in a ring, every rank isends the
sample's messages to its right neighbour and irecvs them from its left one,
then one waitall, several rounds through mpx_enqueue_batch on a persistent
engine.  The configuration with the highest payload rate wins; the table of
every trial comes back with it and can be cached in a JSON file keyed by the
GPU and the sample's signature.  Nothing here moves data itself: each trial
is library calls on device buffers from PyTorch.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

DEFAULT_GRID = {
    "tile_bytes": (16 << 10, 64 << 10, 256 << 10, 1 << 20),
    "bulk_min_bytes": (0, 32 << 10, 256 << 10),
    "engine_ctas": (0, 76),
    "engine_threads": (256, 512),
    "mover_schedule": (0, 1),   # work list / CTA-per-queue (MPX_MOVERS_*)
}


@dataclass
class TuneResult:
    best: Dict[str, int]
    table: List[dict] = field(default_factory=list)
    signature: str = ""


def candidates(grid: Optional[Dict[str, Sequence[int]]] = None) -> List[Dict[str, int]]:
    """Every combination of the grid's values (keys in a fixed order)."""
    g = dict(DEFAULT_GRID if grid is None else grid)
    keys = sorted(g)
    return [dict(zip(keys, vals)) for vals in itertools.product(*(g[k] for k in keys))]


def signature(sizes: Sequence[int], nranks: int) -> str:
    """Key of a message mix: rank count plus a log2-size histogram."""
    hist: Dict[int, int] = {}
    for s in sizes:
        b = max(0, int(s) - 1).bit_length()
        hist[b] = hist.get(b, 0) + 1
    blob = json.dumps({"r": nranks, "h": sorted(hist.items())})
    return hashlib.sha1(blob.encode()).hexdigest()[:16]


def pick(table: List[dict]) -> Dict[str, int]:
    """Highest rate; ties go to the earlier (smaller) configuration."""
    ok = [t for t in table if t.get("ok")]
    if not ok:
        raise RuntimeError("no candidate configuration completed its trial")
    best = max(ok, key=lambda t: (t["gbs"], -ok.index(t)))
    return dict(best["config"])


def _trial(cfg_fields: Dict[str, int], sizes: Sequence[int], nranks: int, rounds: int,
           timeout_s: float) -> dict:
    import numpy as np
    import torch
    from . import mpx
    dev = torch.device("cuda")
    cfg = mpx.mpx_world_config_init()
    for k, v in cfg_fields.items():
        setattr(cfg, k, int(v))
    cfg.max_streams = max(cfg.max_streams, nranks)
    n = len(sizes)
    per_stream = 2 * n + 1
    slots = 256
    while slots < per_stream + 1:
        slots *= 2
    cfg.ring_slots = max(cfg.ring_slots, slots)
    world = mpx.mpx_world_create(nranks, cfg)
    raw = [mpx.mpx_cuda_stream_create() for _ in range(nranks)]
    streams = [mpx.mpx_stream_create(world, r, raw[r], mpx.STREAM_EXCLUSIVE) for r in range(nranks)]
    comm = mpx.mpx_stream_comm_create(world, streams)
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum([(int(s) + 255) // 256 * 256 for s in sizes])
    total = int(offs[-1])
    src = [torch.randint(0, 255, (max(total, 16),), dtype=torch.uint8, device=dev) for _ in range(nranks)]
    dst = [torch.zeros(max(total, 16), dtype=torch.uint8, device=dev) for _ in range(nranks)]
    torch.cuda.synchronize()
    reqs = np.full((nranks, 2 * n), -1, np.int64)
    ops = np.zeros(nranks * (2 * n + 1), mpx.op_dtype())
    k = 0
    for r in range(nranks):
        base = reqs[r].ctypes.data
        for i, s in enumerate(sizes):
            for j, (kind, buf, peer) in enumerate(((mpx.OP_ISEND, src[r], (r + 1) % nranks),
                                                   (mpx.OP_IRECV, dst[r], (r - 1) % nranks))):
                o = ops[k]
                o["kind"], o["datatype"], o["peer"], o["tag"] = kind, mpx.BYTE, peer, i
                o["count"] = int(s)
                o["buf"] = buf.data_ptr() + int(offs[i])
                o["comm"] = comm[r]
                o["requests"] = base + 8 * (2 * i + j)
                k += 1
    for r in range(nranks):
        o = ops[k]
        o["kind"], o["count"], o["requests"] = mpx.OP_WAITALL, 2 * n, reqs[r].ctypes.data
        k += 1
    cs = [torch.cuda.ExternalStream(h, device=dev) for h in raw]
    ok, dt = False, float("inf")
    try:
        mpx.mpx_enqueue_batch(ops)  # warm-up round
        t_dl = time.perf_counter() + timeout_s
        while not all(c.query() for c in cs) and time.perf_counter() < t_dl:
            time.sleep(2e-5)
        t0 = time.perf_counter()
        for _ in range(rounds):
            mpx.mpx_enqueue_batch(ops)
        while not all(c.query() for c in cs) and time.perf_counter() < t_dl:
            time.sleep(2e-5)
        dt = time.perf_counter() - t0
        ok = all(c.query() for c in cs) and mpx.mpx_world_get_error(world) == 0
    finally:
        if not ok:
            mpx.mpx_world_abort(world)
            for c in cs:
                c.synchronize()
        mpx.mpx_world_stop(world, 10000)
        for h in comm:
            mpx.mpx_comm_free(h)
        for s_ in streams:
            mpx.mpx_stream_free(s_)
        mpx.mpx_world_free(world)
        for h in raw:
            mpx.mpx_cuda_stream_destroy(h)
    moved = 2 * sum(int(s) for s in sizes) * nranks * rounds
    return {"config": dict(cfg_fields), "ok": ok, "seconds": dt,
            "gbs": moved / dt / 1e9 if ok else 0.0,
            "msgs_per_s": n * nranks * rounds / dt if ok else 0.0}


def autotune(sizes: Sequence[int], nranks: int = 8, rounds: int = 3,
             grid: Optional[Dict[str, Sequence[int]]] = None, cache: Optional[str] = None,
             timeout_s: float = 30.0,
             trial: Optional[Callable[[Dict[str, int]], dict]] = None) -> TuneResult:
    """Time every candidate on the message mix `sizes` (bytes per message, per
    rank) and return the fastest configuration.  `cache`: a JSON file; a hit
    for this GPU and mix skips the trials, a miss is written back.  `trial`
    replaces the GPU trial (for tests of the selection logic)."""
    sig = signature(sizes, nranks)
    key = sig
    if trial is None:
        import torch
        key = f"{torch.cuda.get_device_name()}|{sig}"
    if cache and os.path.exists(cache):
        with open(cache) as f:
            known = json.load(f)
        if key in known:
            return TuneResult(best=known[key]["best"], table=known[key]["table"], signature=sig)
    run = trial or (lambda c: _trial(c, sizes, nranks, rounds, timeout_s))
    table = [run(c) for c in candidates(grid)]
    res = TuneResult(best=pick(table), table=table, signature=sig)
    if cache:
        known = {}
        if os.path.exists(cache):
            with open(cache) as f:
                known = json.load(f)
        known[key] = {"best": res.best, "table": table}
        with open(cache, "w") as f:
            json.dump(known, f, indent=1)
    return res
