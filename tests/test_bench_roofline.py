"""bench.py's roofline arithmetic on synthetic event timings (no GPU): achieved = algorithmic bytes
or flops / event time, the fraction against the measured or derived peak, the dominant group,
and the DRAM traffic scaled from the ncu bytes per element to one launch."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HBM = 6769.4  # GB/s
N = 4096      # elements per step
STEPS = 5


TF32 = 1697.3 * 1.1 / 2.25  # TFLOP/s


def _tables(prof, work, mode="tf32ir", clk=2070.0):
    return bench.kernel_rooflines(prof, work, STEPS, N, HBM, "measured", mode, clk, tensor_peak=TF32)


def test_contraction_takes_the_binding_roof():
    """The trailing update moves its trailing tiles through HBM and issues each product three times
    on the TF32 pipe: whichever floor binds is its roof.  Here the bytes bind (5.5 TB/s against 66
    TFLOP/s issued): HBM-bound, with the tensor fractions reported beside it."""
    prof = {"lu_tc_update": (96 * 0.456, 96), "gemv": (20.0, 1385)}
    work = {"lu_tc_update": (96 * 2.5e9, 96 * 1.0e10), "gemv": (1385 * 4.8e8, 0.0)}
    kernels, roof = _tables(prof, work)
    assert bench.tensor_peak_tflops({"bf16_tflops": 1893.4, "bf16_tflops_sustained": 1697.3}) == pytest.approx(TF32)
    gbs = 2.5e9 / 0.456e-3 / 1e9
    tflops = 1.0e10 / 0.456e-3 / 1e12
    assert roof["kernel"] == "lu_tc_update" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(gbs) and roof["peak"] == HBM
    assert roof["frac"] == pytest.approx(gbs / HBM)
    assert roof["frac_tensor"] == pytest.approx(tflops / TF32)
    assert roof["frac_tensor_issued"] == pytest.approx(3 * tflops / TF32)
    assert kernels["lu_tc_update"]["bound"] == "hbm"
    # its DRAM counters predate the current update schedule: no traffic figure
    assert "lu_tc_update" not in bench.DRAM_BYTES_PER_ELEMENT_STEP and roof["traffic"] is None


def test_contraction_bound_by_the_tensor_pipe():
    """Ten times fewer bytes, ten times more flops: the issued flops bind (tensor roof), useful
    flops over the TF32 peak derived from the measured sustained BF16 rate."""
    prof = {"lu_tc_update": (96 * 0.456, 96), "gemv": (20.0, 1385)}
    work = {"lu_tc_update": (96 * 2.5e8, 96 * 1.0e11), "gemv": (1385 * 4.8e8, 0.0)}
    kernels, roof = _tables(prof, work)
    tflops = 1.0e11 / 0.456e-3 / 1e12
    assert roof["kernel"] == "lu_tc_update" and roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["achieved"] == pytest.approx(tflops) and roof["peak"] == pytest.approx(TF32)
    assert roof["frac"] == pytest.approx(tflops / TF32)
    assert roof["frac_issued"] == pytest.approx(3 * tflops / TF32)
    assert kernels["lu_tc_update"]["frac_tensor"] == pytest.approx(tflops / TF32)
    assert roof["frac_hbm"] == pytest.approx(2.5e8 / 0.456e-3 / 1e9 / HBM)


def test_hbm_bound_dominant_group():
    # 96 launches of 2.5 GB in 0.456 ms each; the matvec group is smaller
    prof = {"restrict": (96 * 0.456, 96), "gemv": (20.0, 1385), "status": (0.05, 5), "lu_resolve": (0.0, 0)}
    work = {"restrict": (96 * 2.5e9, 96 * 1.0e10), "gemv": (1385 * 4.8e8, 0.0), "status": (1e3, 0.0)}
    kernels, roof = _tables(prof, work)
    assert "lu_resolve" not in kernels                      # no launches: no row
    assert roof["kernel"] == "restrict" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    achieved = 2.5e9 / 0.456e-3 / 1e9
    assert roof["achieved"] == pytest.approx(achieved)
    assert roof["frac"] == pytest.approx(achieved / HBM)
    assert roof["peak"] == HBM
    assert roof["avg_launch_ms"] == pytest.approx(0.456)
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(2.5e9)
    # ncu bytes per element and step, scaled to one of the step's 96 / 5 launches
    per_step = 96 / STEPS
    assert roof["traffic"] == pytest.approx(bench.DRAM_BYTES_PER_ELEMENT_STEP["restrict"] * N / per_step)
    assert kernels["restrict"]["tflops"] == pytest.approx(1.0e10 / 0.456e-3 / 1e12)
    # shares are of all timed groups; "status" (a flag reduction) is timed but has no roofline row
    assert "status" not in kernels
    total = sum(v[0] for v in prof.values())
    assert sum(r["share"] for r in kernels.values()) == pytest.approx(1.0 - prof["status"][0] / total)


def test_alu_bound_dominant_group_uses_the_derived_peak():
    prof = {"residual": (200.0, 10), "restrict": (10.0, 10)}
    work = {"residual": (10 * 5.7e9, 10 * 4.4e13), "restrict": (10 * 6e9, 0.0)}
    kernels, roof = _tables(prof, work)
    assert roof["kernel"] == "residual" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    pk = bench.alu_peak_tflops("ff", "tf32ir", 2070.0)
    # FP32 issue rate 152 x 128 lanes x 2070 MHz; a float-float multiply-add = 12 issue slots for 2 flops
    assert pk == pytest.approx(152 * 128 * 2070e6 * 2 / 12 / 1e12)
    tflops = 4.4e13 / 20e-3 / 1e12
    assert roof["achieved"] == pytest.approx(tflops)
    assert roof["frac"] == pytest.approx(tflops / pk)
    assert kernels["residual"]["frac_alu"] == pytest.approx(tflops / pk)
    assert "tflops" not in kernels["restrict"]


def test_group_without_a_capture_has_no_traffic():
    prof = {"gemv": (120.0, 1385), "krylov": (40.0, 3000)}
    work = {"gemv": (1385 * 4.8e8, 0.0), "krylov": (3000 * 3.7e7, 0.0)}
    _, roof = _tables(prof, work)
    assert roof["kernel"] == "gemv" and roof["traffic"] is None
