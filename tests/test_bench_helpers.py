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
