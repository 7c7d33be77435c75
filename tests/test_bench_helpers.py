"""Host-side helpers of bench.py that shape its JSON line, checked on the CPU:
the clock summary parsed from nvidia-smi samples (median SM clock, maximum,
throttle reasons), the peak figures (measured file or the stated fallback),
the source hash that marks the stored ncu counters fresh or stale, and the
whole-job throughput from the max-over-ranks time."""
import json
import os

import pytest

import bench


def sampler_with(lines):
    c = bench.ClockSampler(0)
    c.lines = list(lines)
    return c


def test_clock_summary_median_max_and_reasons():
    rows = [
        "0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1350.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = sampler_with(rows).summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_thermal_and_hw_slowdown():
    rows = ["0, 1500, 2070, 1400, 0x48, Active, Active, Not Active, Not Active",
            "0, 1600, 2070, 1400, 0x48, Not Active, Not Active, Active, Not Active"]
    s = sampler_with(rows).summary()
    assert s["sm_mhz"] == 1550.0
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = sampler_with([]).summary()
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}


def test_peaks_measured_file_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pk, src = bench.peaks()
    assert src == "fallback" and pk["hbm_gbs"] == 6800.0 and pk["sm_max_mhz"] == 2070.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6782.1,
                                                              "sm_max_mhz": 2070.0}))
    pk, src = bench.peaks()
    assert src == "measured" and pk["hbm_gbs"] == 6782.1


def test_source_hash_marks_counters_fresh_or_stale(tmp_path, monkeypatch):
    """The hash covers the headers whole and, in the .cu file that also holds
    other kernels, only the forward kernel's and its launchers' definitions."""
    csrc = tmp_path / "paper_2511_00292_gb300" / "csrc"
    csrc.mkdir(parents=True)
    cu = None
    for src in bench.FWD_F64_SOURCES:
        if isinstance(src, str):
            (csrc / src).write_text(f"// {src}\n")
        else:
            cu, funcs = src
            body = "".join(f"\n\ntemplate <int L>\nint {f}(int x) {{\n  return x + 1;\n}}\n"
                           for f in funcs)
            other = "\n\nint other_kernel(int y) {\n  return y + k_eigvals<0>(y);\n}\n"
            (csrc / cu).write_text("// unit" + body + other)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_md5(bench.FWD_F64_SOURCES)
    assert h0 == bench.kernel_source_md5(bench.FWD_F64_SOURCES)
    text = (csrc / cu).read_text()
    changed = text.replace("return y +", "return 2 * y +")
    assert changed != text
    (csrc / cu).write_text(changed)                                   # another kernel
    assert bench.kernel_source_md5(bench.FWD_F64_SOURCES) == h0
    (csrc / cu).write_text(text.replace("x + 1", "x + 2", 1))          # the forward kernel
    assert bench.kernel_source_md5(bench.FWD_F64_SOURCES) != h0
    (csrc / cu).write_text(text)
    (csrc / bench.FWD_F64_SOURCES[0]).write_text("// changed header\n")
    assert bench.kernel_source_md5(bench.FWD_F64_SOURCES) != h0


def test_stored_counters_describe_the_committed_source():
    """The per-matrix ncu counters in bench.py were taken on the kernel source
    as committed; a source change without a new capture reports them stale."""
    assert bench.kernel_source_md5(bench.FWD_F64_SOURCES) == bench.FWD_F64_COUNTERS["source_md5"]
    c = bench.FWD_F64_COUNTERS
    assert c["fp64_pipe_inst"] >= c["dfma"] + c["dmul"] + c["dadd"]


def test_whole_job_throughput():
    # 2^28 matrices per GPU, 8 GPUs, 62.8 ms for the slowest rank
    v = bench.weak_scaling_value(8, 1 << 28, 62.8)
    assert v == pytest.approx(8 * (1 << 28) / 0.0628 / 1e9)
    assert bench.weak_scaling_value(1, 1 << 28, 62.8) == pytest.approx(v / 8)
