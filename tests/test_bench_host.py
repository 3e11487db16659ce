"""Host logic of bench.py, without a GPU: the clock sampler's reading of
nvidia-smi samples and throttle reasons, and the rule that a stored DRAM
traffic figure is reported only while its kernel's source is unchanged."""
import hashlib
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Finished:
    """Stands in for an nvidia-smi process that has already exited."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def test_clock_sampler_median_max_and_reasons(tmp_path):
    b = _bench()
    csv = tmp_path / "clocks.csv"
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal,
    # sw_thermal, sw_power_cap (csv, noheader, nounits)
    csv.write_text("0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                   "0, 1980, 2070, 1395.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
                   "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                   "0, [N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "truncated, line\n")
    s = b.ClockSampler(0)
    s.proc, s.path = _Finished(), str(csv)
    r = s.stop()
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert not csv.exists()


def test_clock_sampler_flags_slowdown_reasons(tmp_path):
    b = _bench()
    csv = tmp_path / "clocks.csv"
    csv.write_text("0, 1500, 2070, 1400.0, 0x8, Active, Not Active, Active, Not Active\n"
                   "0, 1600, 2070, 1400.0, 0x8, Not Active, Active, Not Active, Not Active\n")
    s = b.ClockSampler(0)
    s.proc, s.path = _Finished(), str(csv)
    r = s.stop()
    assert r["sm_mhz"] == 1550.0
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    b = _bench()
    r = b.ClockSampler(0).stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_reported_only_for_unchanged_source(tmp_path, monkeypatch):
    b = _bench()
    src = tmp_path / "kernel.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"entries": [{"workload": "w", "kind": "stencil", "source": "kernel.cu",
                        "sha256": hashlib.sha256(src.read_bytes()).hexdigest(), "bytes_per_launch": 12345}]}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(b, "HERE", str(tmp_path))
    assert b._traffic("w", "stencil") == 12345
    assert b._traffic("w", "other") is None
    assert b._traffic("other", "stencil") is None
    src.write_bytes(b"__global__ void k() { /* changed */ }\n")
    assert b._traffic("w", "stencil") is None
    src.unlink()
    assert b._traffic("w", "stencil") is None


def test_committed_traffic_records_are_well_formed():
    # every record names an existing source file, a sha256 and a positive
    # byte count, so that bench.py can check it against the source
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        entries = json.load(f)["entries"]
    assert entries
    for e in entries:
        assert os.path.isfile(os.path.join(ROOT, e["source"])), e["source"]
        assert len(e["sha256"]) == 64 and int(e["sha256"], 16) >= 0
        assert e["bytes_per_launch"] > 0 and e["workload"] and e["kind"] and e["command"]
        assert "--clock-control none" in e["command"]


def test_fp32_alu_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz
    b = _bench()
    assert abs(b.FP32_PEAK_TFLOPS - 80.54784) < 1e-9
