"""Host-side logic of the benchmark that needs no GPU: the clock record taken
during the timed region (median SM clock, throttle reasons), the whole-job
value of one process, the traffic figure tied to the engine source it was
captured from, and the roofline denominator."""
import json
import os

import pytest

bench = pytest.importorskip("bench")


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler()
    s.proc = _FakeProc()
    s.lines = list(lines)
    return s


def test_clock_record_takes_the_median_and_active_reasons(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda _s: None)
    rows = [
        "2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbled line",
        "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    rec = _sampler(rows).stop()
    assert rec["sm_mhz"] == 2055.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples"] == 3


def test_clock_record_reports_thermal_and_hardware_slowdowns(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda _s: None)
    rows = ["1500, 2070, 1200, 0x48, Active, Not Active, Active, Not Active",
            "1490, 2070, 1200, 0x40, Not Active, Active, Not Active, Not Active"]
    rec = _sampler(rows).stop()
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    rec = bench.ClockSampler().stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]


def test_whole_job_of_one_process():
    secs, value = bench.whole_job(2.0, 500)
    assert secs == 2.0 and value == 250.0


def test_traffic_figure_belongs_to_the_captured_engine_source(tmp_path, monkeypatch):
    """The ncu traffic ratio is reported only while the engine source hashes
    to the one captured; any other source gives null."""
    import hashlib
    src = os.path.join(bench.ROOT, "paper_2208_13707_gb300", "csrc", "mpx_engine.cu")
    with open(src, "rb") as f:
        current = hashlib.sha1(f.read()).hexdigest()[:16]
    got = bench.ring_traffic(1000.0)
    if current == bench.RING_TRAFFIC_ENGINE_SHA1:
        assert got == pytest.approx(bench.RING_TRAFFIC_RATIO * 1000.0)
    else:
        assert got is None
    d = tmp_path / "paper_2208_13707_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "mpx_engine.cu").write_bytes(b"// another engine\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ring_traffic(1000.0) is None


def test_peak_is_the_measured_copy_bandwidth(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6781.4}))
    assert bench.peaks() == (6781.4, "measured")
