"""Host logic of bench.py that needs no GPU: the nvidia-smi clock record and
the summary of the forms."""
import os
import sys

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import bench  # noqa: E402


def test_clock_csv_median_max_and_reasons():
    text = "\n".join([
        "2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2040, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",  # a sample that did not parse
        "garbage",
    ])
    c = bench.parse_clock_csv(text)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2040.0
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_csv_thermal_reasons_reported():
    text = ("1500, 2070, 1400.0, 0x48, Active, Active, Not Active, Active\n"
            "1510, 2070, 1400.0, 0x48, Not Active, Not Active, Active, Not Active\n")
    c = bench.parse_clock_csv(text)
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap",
                            "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1505.0


def test_clock_csv_empty():
    c = bench.parse_clock_csv("")
    assert c["samples"] == 0 and c["sm_mhz"] is None and c["reasons"] == []


def test_summary_keys_and_missing_forms():
    assert bench.summarize(1.5, None) == {"tqu16_fp64_solves_s": 1.5}
    forms = {"split_bf16": {"value": 14.6598, "speedup_vs_fp64": 14.8798},
             "qu_nside32": {"split_bf16": {"value": 1.37489}, "fp64": {"value": 0.0478},
                            "split_speedup_vs_fp64": 28.763,
                            "rel_err_split_vs_fp64": {"F": 1.358e-11, "note": "text"}},
             "emulator": {"inference_points_per_s": 2.4381e8}}
    s = bench.summarize(0.98521, forms)
    assert s["tqu16_fp64_solves_s"] == 0.9852
    assert s["tqu16_split_solves_s"] == 14.66
    assert s["qu32_split_speedup"] == 28.76
    assert s["qu32_rel_err_split_vs_fp64"] == {"F": 1.358e-11}  # the note is not a number
    assert s["emu_points_s"] == 2.438e8
    # forms not run are None, not missing
    assert s["scan_split_kt_evals_s"] is None and s["split_gemm_bf16_frac"] is None
    assert s["tqu16_rel_err_fp64"] == {}
