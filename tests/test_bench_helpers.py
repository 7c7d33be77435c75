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


@pytest.mark.parametrize("name", sorted(bench.KERNEL_SOURCES))
def test_source_hash_marks_counters_fresh_or_stale(tmp_path, monkeypatch, name):
    """The hash covers the headers whole and, in the .cu file that also holds
    other kernels, only the kernel's own, its launchers' and its helpers'
    definitions."""
    sources = bench.KERNEL_SOURCES[name]
    csrc = tmp_path / "paper_2511_00292_gb300" / "csrc"
    csrc.mkdir(parents=True)
    cu = None
    for src in sources:
        if isinstance(src, str):
            (csrc / src).write_text(f"// {src}\n")
        else:
            cu, funcs = src
            body = "".join(f"\n\ntemplate <int L>\nint {f}(int x) {{\n  return x + 1;\n}}\n"
                           for f in funcs)
            other = "\n\nint other_kernel(int y) {\n  return y + k_eigvals<0>(y);\n}\n"
            (csrc / cu).write_text("// unit" + body + other)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_md5(sources)
    assert h0 == bench.kernel_source_md5(sources)
    text = (csrc / cu).read_text()
    changed = text.replace("return y +", "return 2 * y +")
    assert changed != text
    (csrc / cu).write_text(changed)                                   # another kernel
    assert bench.kernel_source_md5(sources) == h0
    (csrc / cu).write_text(text.replace("x + 1", "x + 2", 1))          # this kernel
    assert bench.kernel_source_md5(sources) != h0
    (csrc / cu).write_text(text)
    (csrc / sources[0]).write_text("// changed header\n")
    assert bench.kernel_source_md5(sources) != h0


def _strip_comments(text):
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return re.sub(r"//[^\n]*", " ", text)


def _file_level_names(text):
    """Names of the functions and structs defined at file scope of `text`
    (namespace braces do not count as scopes)."""
    import re
    text = _strip_comments(text)
    depth, stack, scope = 0, [], [True] * len(text)
    for i, ch in enumerate(text):
        if ch == "{":
            ns = re.search(r"namespace\s*\w*\s*$", text[max(0, i - 48):i]) is not None
            stack.append(ns)
            depth += 0 if ns else 1
        elif ch == "}":
            depth -= 0 if (stack.pop() if stack else False) else 1
        scope[i] = depth == 0
    names = set()
    for m in re.finditer(r"\bstruct\s+(\w+)\s*\{", text):
        if scope[m.start()]:
            names.add(m.group(1))
    for m in re.finditer(r"\b([A-Za-z_]\w*)\s*\(", text):
        name = m.group(1)
        if not scope[m.start()] or name.startswith("__") or name in ("if", "for", "while"):
            continue
        k, d = m.end() - 1, 0
        for k in range(m.end() - 1, len(text)):   # the parameter list
            d += text[k] == "("
            d -= text[k] == ")"
            if d == 0:
                break
        rest = text[k + 1:k + 64].lstrip()
        if rest.startswith("{") or rest.startswith("const {"):
            names.add(name)
    return names


@pytest.mark.parametrize("name", sorted(bench.KERNEL_SOURCES))
def test_hashed_functions_cover_the_kernel_helpers(name):
    """Every definition of eig3_f64.cu that the kernel or its launchers use
    (directly or through each other) is in the hashed list, so an edit to a
    helper (such as the adjoint-input store) marks the counters stale."""
    import re
    cu, funcs = [s for s in bench.KERNEL_SOURCES[name] if not isinstance(s, str)][0]
    text = open(os.path.join(bench.ROOT, "paper_2511_00292_gb300", "csrc", cu)).read()
    local = _file_level_names(text)
    assert set(funcs) <= local, set(funcs) - local
    seen, todo = set(funcs), list(funcs)
    while todo:
        f = todo.pop()
        for d in bench._definitions(_strip_comments(text), f):
            for used in set(re.findall(r"\b(\w+)\s*[<(]", d)) & local:
                if used not in seen:
                    seen.add(used)
                    todo.append(used)
    assert seen <= set(funcs), f"{name}: not hashed: {sorted(seen - set(funcs))}"


@pytest.mark.parametrize("name", sorted(bench.KERNEL_COUNTERS))
def test_stored_counters_describe_the_committed_source(name):
    """The per-matrix ncu counters in bench.py were taken on the kernel source
    as committed; a source change without a new capture reports them stale."""
    c = bench.KERNEL_COUNTERS[name]
    assert bench.kernel_source_md5(bench.KERNEL_SOURCES[name]) == c["source_md5"]
    assert c["fp64_pipe_inst"] >= c["dfma"] + c["dmul"] + c["dadd"]


# The functions on each kernel's path through eig3_f64.cuh that form binary64
# products on the integer pipes (dmul), with the number of times the kernel
# calls each per matrix.
INT_DMUL_PATH = {
    "vjp_f64_general9": {"invariants_general": 1, "dx13": 2, "triple_angle_sines": 1,
                         "eigvals_vjp_fwd": 1, "adjoint_vjp": 1, "grad_general_vjp": 1},
    "fwd_f64_general9": {"invariants_general": 1, "dx13": 2, "triple_angle_sines": 1,
                         "eigvals_from_inv": 1},
}


@pytest.mark.parametrize("name", sorted(INT_DMUL_PATH))
def test_integer_pipe_products_counted_from_the_source(name):
    """The roofline counts each matrix's integer-pipe products (int_dmul) as
    the dmul call sites on the kernel's path (straight-line code, one
    execution each); every function reached from the path that forms such
    products is on it."""
    import re
    text = _strip_comments(open(os.path.join(bench.ROOT, "paper_2511_00292_gb300", "csrc",
                                             "eig3_f64.cuh")).read())
    path = INT_DMUL_PATH[name]

    def body(f):
        d = bench._definitions(text, f)
        assert len(d) == 1, (f, len(d))
        return d[0]

    defined = {m.group(1) for m in re.finditer(r"__device__[^;{]*?(\w+)\s*\(", text)}

    def forms_dmul(f, seen=()):
        b = body(f)
        return "dmul(" in b or any(forms_dmul(g, seen + (f,)) for g in
                                   set(re.findall(r"\b(\w+)\s*\(", b)) & defined
                                   if g not in seen and g != f and g != "dmul")

    total = sum(k * body(f).count("dmul(") for f, k in path.items())
    assert total == bench.KERNEL_COUNTERS[name]["int_dmul"]
    for f in path:
        for g in set(re.findall(r"\b(\w+)\s*\(", body(f))) & defined - {"dmul", f}:
            assert g in path or not forms_dmul(g), (f, g)


def test_self_launch_command():
    """--gpus N outside torchrun re-runs the same command under
    torch.distributed.run: one rank per GPU, rendezvous on 127.0.0.1."""
    cmd = bench.self_launch_command(4, ["--gpus", "4", "--steps", "5"])
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "--nnodes=1" in cmd
    assert "--master-addr=127.0.0.1" in cmd
    port = int([a for a in cmd if a.startswith("--master-port=")][0].split("=")[1])
    assert 0 < port < 65536
    assert cmd[-4:] == ["--gpus", "4", "--steps", "5"]
    assert cmd[-5].endswith("bench.py")


def test_ratio_stats():
    r = bench.ratio_stats([0.0, 1.0, 2.0, float("nan")], [0.0, 2.0, 1.0, 1.0])
    assert r["max"] == 2.0
    assert bench.ratio_stats([], [])["max"] is None


def test_whole_job_throughput():
    # 2^28 matrices per GPU, 8 GPUs, 62.8 ms for the slowest rank
    v = bench.weak_scaling_value(8, 1 << 28, 62.8)
    assert v == pytest.approx(8 * (1 << 28) / 0.0628 / 1e9)
    assert bench.weak_scaling_value(1, 1 << 28, 62.8) == pytest.approx(v / 8)


def test_kernel_roofline_counts_integer_pipe_products(monkeypatch):
    """The roofline's flop count adds the integer-pipe products to the FP64
    pipe's (FMA = 2), its peak is the two measured peaks added, and every
    figure taken from the counters is null once they are stale."""
    fp = {"fp64_tflops_measured": 1.0, "fp64_tinst_per_s": 0.5, "int_dmul_tops_measured": 0.5,
          "fp32_tflops_measured": 78.0}
    c = dict(bench.KERNEL_COUNTERS["vjp_f64_general9"])
    c.update(dfma=100.0, dmul=10.0, dadd=30.0, int_dmul=60, fp64_warp_inst_x32=140.0,
             fp64_pipe_inst=140.0, dram_bytes=200.0)
    monkeypatch.setitem(bench.KERNEL_COUNTERS, "vjp_f64_general9", c)
    monkeypatch.setattr(bench, "kernel_source_md5", lambda sources: c["source_md5"])
    n, ms = 1 << 20, 1.0
    r = bench.kernel_roofline("vjp_f64_general9", "k", n, ms, fp, 2000.0, 100, 7000.0)
    flop = 2 * 100 + 10 + 30 + 60
    assert r["algorithmic_per_matrix"]["flop"] == flop
    assert r["peak"] == 1.5
    assert abs(r["achieved"] - flop * n / 1e-3 / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / 1.5) < 1e-12
    assert abs(r["frac_vs_fp64_peak"] - r["achieved"] / 1.0) < 1e-12
    assert abs(r["mix_ceiling"] - (2 * 100 + 10 + 30) / (2 * 140.0)) < 1e-12
    assert r["traffic"] == 200.0 * n
    monkeypatch.setattr(bench, "kernel_source_md5", lambda sources: "stale")
    r = bench.kernel_roofline("vjp_f64_general9", "k", n, ms, fp, 2000.0, 100, 7000.0)
    assert not r["counters_fresh"]
    assert all(r[k] is None for k in ("achieved", "frac", "frac_vs_fp64_peak", "traffic"))
