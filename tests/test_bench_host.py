"""Host logic of the benchmark, without a GPU: the clock-record summary (median clock and
throttle reasons from nvidia-smi rows), the CPU oracle sample that serves as the reported
baseline, and the reference arm's JSON line."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_clock_summary_reports_median_and_reasons():
    cs = bench.ClockSampler(0)
    row = lambda mhz, thermal: ["0", str(mhz), "2070", "900.0", "0x0", "Not Active",  # noqa: E731
                                "Active" if thermal else "Not Active", "Not Active", "Active"]
    cs.rows = [row(2070, False), row(1980, False), row(2070, True), ["garbage"]]
    out = cs.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_oracle_sample_is_a_bounded_cpu_baseline():
    out = bench.oracle_sample(seconds_target=0.05, n=2, slabs=2)
    assert out["kind"] == "oracle" and out["cores"] == 1 and out["unit"] == "DoF/s"
    assert out["value"] > 0 and out["seconds"] > 0 and "2^3 hexes" in out["sample"]


def test_reference_arm_line(capsys, monkeypatch):
    fake = {"value": 1000.0, "unit": "DoF/s", "cores": 1, "kind": "oracle", "seconds": 2.0, "sample": "s"}
    monkeypatch.setattr(bench, "oracle_sample", lambda **kw: dict(fake))

    class A:
        steps, warmup, gpus, n, r, slabs = 2, 1, 1, 32, 1, 16
    assert bench.run_reference(A) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] == 1000.0 and line["ms_per_step"] == 2000.0
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert "32^3 hexes" in line["config"]["workload"]
