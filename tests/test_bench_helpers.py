"""Host-side arithmetic of bench.py's ALU roofline."""
import pytest


def test_alu_flops_per_voxel():
    import bench
    from paper_1907_02731_gb300 import inputs
    wl = inputs.WORKLOADS["video_72x480x854"]
    # 3 pre-products, 3 x (5 + 11 + 11) FMAs, 8 combine, 10 reduction flops
    assert bench.alu_flops_per_voxel(wl) == 3 + 2 * 3 * 27 + 8 + 10
    wl2 = inputs.WORKLOADS["video2ch_72x480x854"]
    assert wl2.nchan == 2
    assert bench.alu_flops_per_voxel(wl2) == 5 + 2 * 4 * 27 + 16 + 10


def test_clock_summary_parses_samples_and_reasons():
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2040, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and "window" not in s
    c.after = True                     # only a sample taken after a short timed region
    assert "first sample after" in c.summary()["window"]
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_dram_traffic_is_keyed_to_the_kernel_sources(monkeypatch):
    """The recorded DRAM bytes are reported only for the kernel sources they
    were captured on; any change to those sources turns them into null."""
    import bench
    rec = bench.DRAM_TRAFFIC_PER_LAUNCH[("video_72x480x854", "f32")]
    monkeypatch.setattr(bench, "kernel_hash", lambda: rec[1])
    assert bench.dram_traffic("video_72x480x854", "f32") == (rec[0], None)
    assert bench.dram_traffic("small_16x64x64", "f32") == (None, "not captured for this workload")
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.dram_traffic("video_72x480x854", "f32") == (None, "kernel changed since the capture")

