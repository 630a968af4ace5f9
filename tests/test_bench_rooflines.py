"""Host logic of the bench (CPU): the bound, peak and achieved rate of every kernel class are
formed from the timers' (ms, algorithmic work, launches) as the design notes state them, the
dominant class becomes the roofline entry, and the nvidia-smi clock samples are summarised."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Solver:
    """Stand-in for the handle: two substructures with 100 and 200 interface dofs."""
    nsub = 2
    precision = 1

    def interface_dofs(self, i):
        return np.arange(100 if i == 0 else 200)


def test_kernel_table_bounds_and_rates():
    bf16, hbm, _ = bench._peaks()
    steps = 2
    kt = {
        "oz_syrk_bf16": (20.0, 4e12, 10),      # ms, effective flop, launches over the timed steps
        "pcg_kernel": (10.0, 0.0, 2),
        "tc_gemm_3xtf32": (4.0, 1e12, 4),
        "pchol_update_ff": (6.0, 3e11, 8),
        "oz_split": (3.0, 0.0, 10),
        "face_reduction": (0.0, 0.0, 0),       # no launches: left out
    }
    out = bench._kernel_table(kt, steps, _Solver(), {"iters": 30}, "irregular48")
    assert "face_reduction" not in out
    oz = out["oz_syrk_bf16"]
    assert oz["bound"] == "tensor" and oz["peak"] == bf16
    # 28 executed digit products per effective multiply-add, per launch, over the mean launch time
    assert abs(oz["achieved"] - 28 * 4e12 / 10 / (20.0 / 10 / 1e3) / 1e12) < 1e-9 * oz["achieved"]
    assert abs(oz["frac"] - oz["achieved"] / bf16) < 1e-12
    assert oz["traffic"] == bench.TRAFFIC[("irregular48", "oz_syrk_bf16")]   # measured DRAM bytes per launch
    assert out["pcg_kernel"]["traffic"] is None                              # not measured: null
    pcg = out["pcg_kernel"]
    # one FP64 multiply-add per 8-byte entry of S_i and P~_i: the FP64 pipe caps the stream below HBM
    fp64_gbs = bench.PEAK_FP64_TFLOPS * 1e12 / 2 * 8 / 1e9
    assert pcg["bound"] == ("alu" if fp64_gbs < hbm else "hbm")
    assert abs(pcg["peak"] - min(fp64_gbs, hbm)) < 1e-9 * pcg["peak"]
    b = 2 * 8 * (100 ** 2 + 200 ** 2) * 30
    assert pcg["work_per_launch"] == b
    assert abs(pcg["achieved"] - b / (10.0 / 2 / 1e3) / 1e9) < 1e-9 * pcg["achieved"]
    tc = out["tc_gemm_3xtf32"]
    assert tc["bound"] == "tensor"
    assert abs(tc["peak"] - bf16 * bench.NOMINAL_TF32_OVER_BF16) < 1e-9
    ff = out["pchol_update_ff"]
    assert ff["bound"] == "alu" and ff["peak"] == bench.PEAK_FF_TFLOPS
    assert out["oz_split"]["bound"] == "latency"
    for e in out.values():
        assert abs(e["ms_per_step"] * steps - kt[e["kernel"]][0]) < 1e-12
    entry = bench._roofline_entry(max(out.values(), key=lambda e: e["ms_per_step"]))
    assert entry["kernel"] == "oz_syrk_bf16" and set(("bound", "achieved", "peak", "frac")) <= set(entry)


def test_derived_peaks():
    # 152 SMs at 2.07 GHz: FP64 4 flop, FP32 2 x 128 lanes, double-float 12 FP32 instructions per
    # multiply-add (2 FP64-equivalent flop)
    assert abs(bench.PEAK_FP64_TFLOPS - 1.25856) < 1e-9
    assert abs(bench.PEAK_FP32_TFLOPS - 80.54784) < 1e-9
    assert abs(bench.PEAK_FF_TFLOPS - 6.71232) < 1e-9


def test_clock_samples_summary():
    # columns: index, clocks.sm, clocks.max.sm, power.draw, active reasons (bit mask), hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    lines = [
        "0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.7, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped
        "0, 2070, 2070",                                                                  # short: skipped
        "0, 2055, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.parse_clocks(lines)
    assert c == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.parse_clocks(["0, 1500, 2070, 1400, 0x48, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.parse_clocks([]) is None and bench.parse_clocks(["garbage"]) is None
