"""The bench's accounting on the host: the push launch's roofline from the
device's work counts, the cells the field kernels updated, and the clock
record.  Pure arithmetic on fabricated counts; no GPU.

The push's roofline divides by work the device counted in the timed window
(full pushes and quiet drifts), so a window in which the quiet-tile pass moved
every ion reports no FP32 work at all, whatever its bytes; these tests fix
that arithmetic by hand-worked numbers."""
import json
import math
import os

import bench


def test_quiet_window_reports_no_fp32_work():
    # one launch, 1 ms, only quiet drifts: zero FP32 operations, bytes of the
    # drifts (68 B) plus the per-cell field and current bytes (36 B)
    r = bench.push_roofline(0, 1_000_000, 1, 1.0, 1000, 6000.0, "measured", 2000.0, sms=100)
    assert r["achieved"] == 0.0 and r["frac"] == 0.0
    assert r["hbm"]["bytes_per_launch"] == 68_000_000 + 36_000
    assert math.isclose(r["hbm"]["achieved"], 68.036, rel_tol=1e-12)  # GB/s over 1 ms
    assert math.isclose(r["hbm"]["frac"], 68.036 / 6000.0, rel_tol=1e-12)


def test_full_pushes_set_the_fp32_roof():
    # two launches of 2 ms in all (1 ms each), 2e6 full pushes in all: 1e6 per
    # launch x 2371 flops in 1 ms = 2.371 TFLOP/s; peak 100 SMs x 128 x 2 x 2 GHz
    r = bench.push_roofline(2_000_000, 0, 2, 2.0, 0, 6000.0, "measured", 2000.0, sms=100)
    assert math.isclose(r["peak"], 51.2, rel_tol=1e-12)
    assert math.isclose(r["achieved"], 2.371, rel_tol=1e-12)
    assert math.isclose(r["frac"], 2.371 / 51.2, rel_tol=1e-12)
    assert r["hbm"]["bytes_per_launch"] == 1_000_000 * 104
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"


def test_traffic_scales_the_measured_bytes_per_ion_by_the_counted_work():
    r = bench.push_roofline(300, 500, 1, 1.0, 0, 6000.0, "measured", 2000.0, sms=100)
    assert math.isclose(r["traffic"], 300 * bench.TRAFFIC_FULL_ION + 500 * bench.TRAFFIC_QUIET_ION,
                        rel_tol=1e-12)


def test_gb300_fp32_peak_from_unit_counts():
    # 152 SMs x 128 lanes x 2 flops x 2070 MHz
    peak, sms = bench.fp32_peak_tflops(2070.0, 152)
    assert sms == 152 and math.isclose(peak, 80.54784, rel_tol=1e-12)


def test_zero_launches_do_not_divide_by_zero():
    r = bench.push_roofline(0, 0, 0, 1.0, 10, 6000.0, "measured", 2000.0, sms=1)
    assert r["frac"] == 0.0 and r["hbm"]["bytes_per_launch"] == 360


def test_updated_cells_with_and_without_tile_flags():
    # 16 tiles of 4 cells: 10 tile updates counted over 5 flagged steps
    assert bench.updated_cells(10, 5, 64, 16, 5) == 40
    # a grid that keeps no flags updates every cell every step
    assert bench.updated_cells(0, 0, 64, 16, 5) == 320


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.0, 0x0, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_and_reasons():
    lines = [_line(2070, 2070), _line(1900, 2070, cap="Active"), _line(2000, 2070),
             "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
             "garbage"]
    c = bench.summarize_clocks(lines)
    assert c["samples"] == 3 and c["sm_mhz"] == 2000.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_hardware_slowdowns():
    c = bench.summarize_clocks([_line(1500, 2070, hw="Active"), _line(1400, 2070, swt="Active"),
                                _line(1450, 2070, hwt="Active")])
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_of_no_samples():
    c = bench.summarize_clocks([])
    assert c["sm_mhz"] is None and c["samples"] == 0 and c["reasons"] == []


def test_peaks_read_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1234.5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (1234.5, "measured")
    os.remove(tmp_path / "MEASURED_PEAKS.json")
    assert bench.peaks() == (6800.0, "fallback")


def test_single_process_whole_job_is_the_local_figures():
    assert bench.whole_job(12.5, 7) == (12.5, 7.0)
