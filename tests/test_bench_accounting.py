"""Host-side accounting of bench.py: the algorithmic operations and bytes per cell-stage that the
roofline fractions divide by, checked against the per-kernel figures stated with the rooflines
(TENO5 reconstruction 78 operations, WENO5-JS 68; a convective pass 831 / 731 per cell; 2691 in
a 3D viscous TENO5 stage; 106.7 B per cell-stage for a fused FP64 stage) and for consistency
between 2D and 3D."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_operation_counts_3d():
    t = bench.flops_per_cell("teno5")
    w = bench.flops_per_cell("weno5js")
    assert t["conv_x"] == t["conv_y"] == t["conv_z"] == 831
    assert w["conv_x"] == 731
    assert (t["pad"], t["visc_flux"], t["visc_div"], t["finish"]) == (17, 80, 76, 25)
    assert t["total"] == 2691
    assert t["total"] - w["total"] == 3 * 100   # 10 per reconstruction, 2 x 5 per face, 3 passes


def test_operation_counts_2d_and_inviscid():
    t2 = bench.flops_per_cell("teno5", dim=2)
    assert t2["conv_z"] == 0
    # 4 components: two reconstructions of 78 and their sum per component
    assert t2["conv_x"] == (2 + 3) + 5 * 4 + 4 * (2 * 78 + 1) + 3 * 4
    inv = bench.flops_per_cell("teno5", viscous=False)
    assert inv["visc_flux"] == inv["visc_div"] == 0
    assert inv["total"] == 2691 - 80 - 76


def test_fused_stage_bytes():
    assert math.isclose(bench.bytes_per_cell_stage(3), 320.0 / 3.0)
    assert math.isclose(bench.bytes_per_cell_stage(2), 0.8 * 320.0 / 3.0)


def test_fp32_finish_bytes_by_stage_mean():
    # stage 1: L 20, velocity perturbations 12, increment out 20; stage 2: + increment in 20;
    # stage 3: increment in 20, FP64 state read and written 80, FP32 copy 20 -> mean 92 B
    b = bench.bytes_per_cell("fp32")
    assert math.isclose(b["finish"], 92.0)


class _Fake:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def join(self, timeout=None):
        pass


def test_clock_record_parsing():
    c = object.__new__(bench.Clocks)
    c.proc, c.th = _Fake(), _Fake()
    row = "0, {sm}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {cap}"
    c.rows = [[x.strip() for x in row.format(sm=sm, cap=cap).split(",")]
              for sm, cap in ((2070, "Not Active"), (1980, "Active"), (2070, "Not Active"))]
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    # no sampler at all: stated, not silently empty
    c2 = object.__new__(bench.Clocks)
    c2.proc = None
    assert c2.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_stage_roofline_is_the_whole_stage_unit():
    # 512^3 cells, 13.04 ms per stage: 106.7 B x 1.342e8 / 13.04 ms = 1.098 TB/s
    cells = 512 ** 3
    r = bench.stage_roofline(bench.bytes_per_cell_stage(), cells, 13.04, 6787.6, "measured",
                             2691, 80.5, None)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert math.isclose(r["achieved"], 320.0 / 3.0 * cells / 13.04e-3 / 1e9)
    assert math.isclose(r["frac"], r["achieved"] / 6787.6)
    assert 0.16 < r["frac"] < 0.17
    assert math.isclose(r["alu_frac"], 2691 * cells / 13.04e-3 / 1e12 / 80.5)
