"""Host-side logic of bench.py that its numbers rest on (no GPU): the stored
DRAM traffic is used only while the kernel sources it was measured on are
unchanged (comments aside), the algorithmic bytes per cell-stage, the
roofline arithmetic, and the clock-record parsing that decides whether a
run is kept."""
import json

import pytest

import bench


def test_stored_traffic_is_used_only_for_unchanged_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1812_04135_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    k = csrc / "k.cu"
    k.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"dram_bytes_per_launch": 1234, "sources": ["k.cu"], "sources_sha": bench._sources_sha(["k.cu"])}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"w:fp64:8": entry}))
    assert bench._traffic_key("w:fp64:8") == 1234
    assert bench._traffic_key("no:such:workload") is None
    k.write_text("__global__ void k() { int x = 1; }\n")   # the kernel changed: the stored figure is stale
    assert bench._traffic_key("w:fp64:8") is None


def test_sources_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1812_04135_gb300" / "csrc"
    csrc.mkdir(parents=True)
    f = csrc / "k.cu"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    f.write_text("int a = 1;  // one\n/* block */\nint b = 2;\n")
    h0 = bench._sources_sha(["k.cu"])
    f.write_text("int a = 1;  // first\n\n/* another\n block */\nint b = 2;   \n")
    assert bench._sources_sha(["k.cu"]) == h0
    f.write_text("int a = 1;\nint b = 3;\n")
    assert bench._sources_sha(["k.cu"]) != h0


def test_algorithmic_bytes_per_cell_stage():
    # 2.5 nvar s: 2D float64 80 B, 3D float64 100 B, 2D float32 40 B, 1D float64 60 B
    assert bench.bytes_per_cell_stage({"ndim": 2}, "fp64") == 80.0
    assert bench.bytes_per_cell_stage({"ndim": 3}, "fp64") == 100.0
    assert bench.bytes_per_cell_stage({"ndim": 2}, "fp32_pert") == 40.0
    assert bench.bytes_per_cell_stage({"ndim": 1}, "fp64_df") == 60.0


def test_roofline_objects(monkeypatch):
    """achieved = algorithmic bytes (or flops) per launch / launch time; frac
    = achieved / peak; the float64 peak is the measured probe's."""
    monkeypatch.setattr(bench, "fp64_peak_measured", lambda dev: (1.2, 300.0, 2070.0))
    peaks = {"hbm_gbs": 6000.0}
    h = bench._roof_hbm({"ndim": 2}, "fp32_pert", 1000, 1e-6, peaks, "measured", None)
    assert h["achieved"] == pytest.approx(40 * 1000 / 1e-6 / 1e9) and h["frac"] == pytest.approx(h["achieved"] / 6000.0)
    a = bench._roof_alu(309, 1000, 1e-6, None, "count")
    assert a["achieved"] == pytest.approx(309 * 1000 / 1e-6 / 1e12) and a["peak"] == 1.2
    assert a["frac"] == pytest.approx(a["achieved"] / 1.2)


def test_clock_record_from_nvidia_smi_lines():
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_record_from_nvml_samples():
    c = bench.ClockSampler(0)
    c.nvml = object()          # the summary only checks that NVML was used
    c.max_mhz = 2070.0
    c.samples = [(2070.0, 0x0), (2070.0, 0x4), (1800.0, 0x8 | 0x40)]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
