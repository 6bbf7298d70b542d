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


def test_schur_roofline_and_dominant_kernel_choice():
    # 10 launches, 0.3 ms in all, 3e7 point x column units, 8 MB of weights per launch, a 2 ms step
    r = bench.schur_roofline((10, 0.3, 3e7), 8e6, 0.002, 6700.5, traffic_per_unit=20.5, traffic_file="f")
    alg = 20.0 * 3e7 + 8e6 * 10
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - alg / 0.3e-3 / 1e9) < 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 6700.5) < 1e-15
    assert abs(r["traffic"] - 20.5 * 3e6) < 1e-6 and r["traffic_source"]
    assert abs(r["share_of_step"] - 0.15) < 1e-15 and abs(r["avg_launch_us"] - 30.0) < 1e-12
    assert bench.schur_roofline((0, 0.0, 0.0), 8e6, 2.0, 6700.5) is None
    el = {"kernel": "elasticity", "share_of_step": 0.2}
    first, second = bench.dominant_roofline(el, r)
    assert first is el and second is r
    first, second = bench.dominant_roofline(dict(el, share_of_step=0.1), r)
    assert first is r and second["kernel"] == "elasticity"
    # profiling off: no shares, the first object is kept
    none = {"kernel": "elasticity", "share_of_step": None}
    assert bench.dominant_roofline(none, None) == (none, None)


def test_profile_figures_are_read_from_the_committed_summaries():
    assert bench.profile_figure("elasticity_fp32_64cube.txt", "dram_bytes_per_node_rhs:") > 24.0
    assert bench.profile_figure("schur_step_fp32_64cube.txt", "dram_bytes_per_point_rhs:") > 4.0
    assert bench.profile_figure("absent.txt", "x:") is None
