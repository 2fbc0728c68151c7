"""Host logic of bench.py that needs no GPU: the DRAM traffic taken from the
committed ncu summary (scaled to the lattice, and dropped once the kernel
source no longer matches the capture), the clock summary of the nvidia-smi
samples, and the roofline arithmetic of the headline line."""
import os

import pytest

import bench


def test_traffic_is_read_from_the_committed_summary():
    txt = open(bench.PROFILE).read()
    assert "kernel_source_sha256_16" in txt and "dram_bytes_per_cell" in txt
    got = bench._traffic_per_launch(1000)
    if got is None:
        pytest.skip("the step kernel changed since the ncu capture; its traffic is reported as null")
    per_cell = got / 1000
    # the capture's DRAM bytes per update lie within a few percent of the 360 B the step moves
    assert 0.97 * bench.BYTES_MOVED_PER_UPDATE < per_cell < 1.10 * bench.BYTES_MOVED_PER_UPDATE


def test_traffic_is_null_once_the_kernel_changes(tmp_path, monkeypatch):
    src = tmp_path / "lb_kernels.cuh"
    src.write_bytes(open(bench.KERNEL_SRC, "rb").read() + b"\n// edited\n")
    monkeypatch.setattr(bench, "KERNEL_SRC", str(src))
    assert bench._traffic_per_launch(1000) is None


def test_traffic_scales_with_the_cells_of_a_launch(tmp_path, monkeypatch):
    prof = tmp_path / "p.md"
    prof.write_text("- kernel_source_sha256_16: `%s`\n- dram_bytes_per_cell: 371.5\n" % bench._kernel_hash())
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench._traffic_per_launch(4096 * 4096) == pytest.approx(371.5 * 4096 * 4096)
    prof.write_text("- kernel_source_sha256_16: `%s`\n" % bench._kernel_hash())
    assert bench._traffic_per_launch(10) is None


def test_clock_summary_median_max_and_reasons():
    c = bench.ClockSampler(0)
    c.rows = [["2070", "2070", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["1980", "2070", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["2040", "2070", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["[N/A]", "2070", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4
    c.rows = [["2070", "2070", "0x8", "Active", "Not Active", "Active", "Not Active"]]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["no samples"]


def test_roofline_fraction_arithmetic():
    # the algorithmic 352 B per update (36 populations and 8 lagged fields, read
    # and written) at 13.44 GLUPS is 4.73 TB/s: 0.698 of a 6778.7 GB/s copy peak
    assert bench.BYTES_PER_UPDATE == 36 * 4 * 2 + 8 * 4 * 2
    achieved = bench.BYTES_PER_UPDATE * 13439.41e6 / 1e9
    assert achieved == pytest.approx(4730.7, abs=0.1)
    assert achieved / 6778.7 == pytest.approx(0.6979, abs=1e-4)
    assert achieved / bench.NAMEPLATE_HBM_GBS == pytest.approx(0.5988, abs=1e-4)
    assert bench.BYTES_PER_UPDATE_F16 == 36 * 2 * 2 + 8 * 4 * 2
    assert bench.BYTES_PER_UPDATE_Q5 == 28 * 4 * 2 + 8 * 4 * 2
    assert bench.BYTES_PER_UPDATE_F16H == 27 * 2 * 2 + 9 * 4 * 2 + 8 * 4 * 2


def test_peaks_fall_back_when_the_measured_file_is_absent(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, source = bench._peaks()
    assert source == "fallback" and peaks["hbm_gbs"] == 6800.0
    if os.path.exists(os.path.join(os.path.dirname(bench.__file__), "MEASURED_PEAKS.json")):
        monkeypatch.undo()
        assert bench._peaks()[1] == "measured"
