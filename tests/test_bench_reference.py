"""The benchmark's reference arm (the FP64 oracle on the host cores) runs without a GPU and
prints one JSON line with the fields the benchmark contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-pixels", "24"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "queries/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_cpu_baseline_is_the_reference_measurement():
    """The GPU arm's cpu_baseline is the reference arm's own measurement, run in a fresh
    process after every oracle pyramid level was built (so no timed step builds one)."""
    sys.path.insert(0, ROOT)
    import bench
    cb = bench.cpu_baseline_subprocess(24, 2, 1)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1
    assert cb["per_step_min"] <= cb["per_step_median"] <= cb["per_step_max"]
    assert "pyramid level built first" in cb["sample"]


def test_clock_sampler_summarises_nvml_samples(monkeypatch):
    """The timed-region clock record from a fake NVML (no GPU): median SM clock, maximum,
    sample count and the union of the clock event reasons seen."""
    sys.path.insert(0, ROOT)
    import time
    import bench

    class FakeNvml:
        def __init__(self):
            self.n = 0

        def sample(self):
            self.n += 1
            return (1980.0, 2070.0, ["sw_power_cap"]) if self.n % 2 else (2070.0, 2070.0, [])

    monkeypatch.setattr(bench._Nvml, "open", classmethod(lambda cls, index: FakeNvml()))
    c = bench.Clocks(0)
    c.start()
    time.sleep(0.05)
    rec = c.stop()
    assert rec["samples"] >= 3 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"] and 1980.0 <= rec["sm_mhz"] <= 2070.0
    assert rec["sm_mhz_min"] == 1980.0


def test_clock_sampler_without_nvml_or_nvidia_smi(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench._Nvml, "open", classmethod(lambda cls, index: None))
    monkeypatch.setenv("PATH", "/nonexistent")
    c = bench.Clocks(0)
    c.start()
    assert c.stop() is None
