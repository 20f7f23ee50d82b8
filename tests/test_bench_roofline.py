"""Host-side arithmetic of the bench line's roofline (no GPU): the dominant stage is the
slowest one, its bound is the roof it is closer to, and the fractions are the algorithmic
work over the stage time over the measured peaks."""
import math

import bench


def test_roofline_dominant_stage_bound_and_fractions():
    peaks = {"fp64": 1.25e12, "fp32": 73.0e12}
    hbm, _ = bench.hbm_peak_gbs()
    stage_ms = {"p2p": 50.0, "m2x": 20.0, "x2x": 10.0, "gather": 0.0}
    work = {"p2p": (40e9, 7.2e7), "m2x": (10e9, 4e9), "x2x": (1e9, 30e9)}
    r = bench.roofline("fp64", stage_ms, work, peaks, n_beads=1_000_000)
    assert r["kernel"] == "p2p" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert math.isclose(r["achieved"], 40e9 / 0.05 / 1e12, rel_tol=1e-3)
    assert math.isclose(r["frac"], 40e9 / 0.05 / 1.25e12, rel_tol=1e-3)
    # FP64 near field: traffic from the per-bead capture figure, scaled by the bead count
    assert r["traffic"] == round(bench.P2P64_DRAM_BYTES_PER_BEAD * 1_000_000)
    st = r["stages"]
    assert "gather" not in st   # a stage of zero time has no rate
    assert math.isclose(st["x2x"]["frac_hbm"], 30e9 / 0.01 / 1e9 / hbm, rel_tol=1e-3)
    assert math.isclose(st["m2x"]["frac_alu"], 10e9 / 0.02 / 1.25e12, rel_tol=1e-3)


def test_roofline_hbm_bound_and_fp32_peak():
    peaks = {"fp64": 1.25e12, "fp32": 73.0e12}
    hbm, _ = bench.hbm_peak_gbs()
    stage_ms = {"x2l": 4.0, "p2p": 1.0}
    work = {"x2l": (1e9, 20e9), "p2p": (5e9, 1e7)}
    r = bench.roofline("fp32", stage_ms, work, peaks)
    assert r["kernel"] == "x2l" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert math.isclose(r["frac"], 20e9 / 0.004 / 1e9 / hbm, rel_tol=1e-3)
    assert r["traffic"] is None   # no capture figure for this kernel
    assert math.isclose(r["stages"]["p2p"]["frac_alu"], 5e9 / 0.001 / 73.0e12, rel_tol=1e-3)
