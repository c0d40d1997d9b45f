"""Autotuner: candidate grid, mix signature, selection and cache (CPU, with a
fake trial), and one small real tuning run on the GPU."""
import json

import pytest

from paper_2208_13707_gb300 import autotune as at


def test_grid_is_the_cartesian_product():
    c = at.candidates({"tile_bytes": (1, 2), "engine_ctas": (0, 76, 38)})
    assert len(c) == 6
    assert {tuple(sorted(x.items())) for x in c} == {
        (("engine_ctas", e), ("tile_bytes", t)) for e in (0, 76, 38) for t in (1, 2)}


def test_signature_depends_on_the_size_histogram_and_ranks():
    a = at.signature([100, 200, 4096], 8)
    assert a == at.signature([120, 250, 4000], 8)      # same power-of-two bins
    assert a != at.signature([100, 200, 8193], 8)
    assert a != at.signature([100, 200, 4096], 16)


def test_pick_takes_the_fastest_completed_trial_and_caches(tmp_path):
    rates = {16: 5.0, 64: 9.0, 256: 7.0}

    def fake(cfg):
        ok = cfg["engine_ctas"] == 0
        return {"config": cfg, "ok": ok, "gbs": rates[cfg["tile_bytes"]] if ok else 99.0}

    grid = {"tile_bytes": (16, 64, 256), "engine_ctas": (0, 76)}
    cache = tmp_path / "tune.json"
    r = at.autotune([64, 1 << 20], grid=grid, cache=str(cache), trial=fake)
    assert r.best == {"engine_ctas": 0, "tile_bytes": 64}     # failed trials never win
    assert len(r.table) == 6
    calls = []
    r2 = at.autotune([64, 1 << 20], grid=grid, cache=str(cache),
                     trial=lambda c: calls.append(c) or fake(c))
    assert r2.best == r.best and not calls                      # served from the cache
    assert json.loads(cache.read_text())[r.signature]["best"] == r.best
    with pytest.raises(RuntimeError):
        at.pick([{"config": {}, "ok": False, "gbs": 1.0}])


@pytest.mark.gpu
def test_autotune_runs_on_the_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    grid = {"tile_bytes": (16 << 10, 64 << 10), "bulk_min_bytes": (0, 32 << 10),
            "engine_ctas": (0,), "engine_threads": (256,)}
    sizes = [8, 512, 4096, 65536, 1 << 20, 4 << 20]
    r = at.autotune(sizes, nranks=4, rounds=2, grid=grid)
    assert all(t["ok"] for t in r.table), r.table
    assert r.best in [t["config"] for t in r.table]
    assert max(t["gbs"] for t in r.table) > 0
