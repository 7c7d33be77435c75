"""Benchmark: batched stable closed-form 3x3 eigenvalues on GB300.

One step = one forward + backward pass of the whole path over the mixed
workload of 2^28 matrices per GPU: 2^27 symmetric 6-entry binary32 matrices
through the compensated binary32 kernel and 2^27 general 9-entry binary64
matrices through the binary64 kernel (invariants I1, J2, J3, Delta ->
triple angle -> eigenvalues -> adjoint, fused in one pass per matrix:
eig3_eigvals_vjp), the two halves on two streams.
Inputs are resident in HBM and larger than L2 (about 18 GB per step), so no
L2 flush is needed between steps.

Printed (rank 0, one JSON line): whole-job throughput in G matrices/s, the
roofline of the dominant kernel (the fused binary64 kernel) and of the
binary64 forward, both against peaks measured in the same run by throughput
loops (the FP64 pipe's DFMA rate plus the rate of the binary64 products the
kernels form on the integer pipes; the FP32 rate beside them), per-path throughputs of the other workloads' shapes (among
them the step as one CUDA graph of 10 steps, and unfused), the CPU oracle
timed on the host cores on a bounded sample (with the max error over the
stability bound of the GPU results on that sample, and the distance of the
GPU results from the exact eigenvalues and invariants per eigenvalue and
per invariant), an end-to-end number through host buffers, and SM clocks
sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --peaks            (the FP64 / FP32 / integer-pipe product peaks alone)
  python bench.py --only KERNEL --n N (one kernel alone, for profiler captures)
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "G matrices/s fwd and fwd+bwd (FP64 vs FP32-comp) vs roofline; max err/stab bound"
UNIT = "G matrices/s"
N_MIXED = 1 << 28
WORKLOAD = ("mixed fwd+bwd, 2^28 matrices/GPU: 2^27 symmetric 6-entry FP32 (compensated FP32 "
            "path) + 2^27 general 9-entry FP64 (FP64 path), scales 10^U[-8,8], 30% "
            "triple-perturbed; loss sum(w lambda), w ~ N(0,1); forward and vector-Jacobian "
            "product fused per half, the binary32 half on a second stream")

# Per-matrix ncu counters of the two binary64 kernels whose rooflines the line
# reports, each taken with ncu on n = 2^22 (bench.py --only NAME, the same
# launch as in the timed step): thread-level instructions on the FP64 pipe
# (active lanes only) and the warp-level count times 32 (what occupies the
# pipe, idle lanes included), of which DFMA / DMUL / DADD, and DRAM bytes read
# + written; int_dmul is the number of binary64 products each matrix forms on
# the integer pipes (dmul call sites on the kernel's path, one execution each;
# tests/test_bench_helpers.py counts them in the source).  They describe the
# kernel source whose
# hash is recorded; when the source changes they are reported as stale and
# every figure derived from them as null.
KERNEL_COUNTERS = {
    "vjp_f64_general9": {
        "source_md5": "1c9c3e78e86efc45d5e7114fec5f325e",
        "fp64_pipe_inst": 144.02, "fp64_warp_inst_x32": 144.50,
        "dfma": 105.01, "dmul": 5.00, "dadd": 34.01, "int_dmul": 68,
        "dram_bytes": (404.403712e6 + 351.489280e6) / 4194304,
    },
    "fwd_f64_general9": {
        "source_md5": "6814059c5f439f9e4b45703914d9560f",
        "fp64_pipe_inst": 108.00, "fp64_warp_inst_x32": 108.00,
        "dfma": 79.00, "dmul": 7.00, "dadd": 22.00, "int_dmul": 47,
        "dram_bytes": (302.136832e6 + 189.932544e6) / 4194304,
    },
}
# What each hash covers: the headers whole and, of eig3_f64.cu (which holds
# other kernels too), the kernel's own definitions, its launchers and every
# helper of that file they use (tests/test_bench_helpers.py checks the list
# against the kernel bodies).
KERNEL_SOURCES = {
    "vjp_f64_general9": ("eig3_f64.cuh", "eig3_dmul.cuh", "eig3_stats.cuh", "eig3_tile.cuh",
                         ("eig3_f64.cu", ("k_eigvals_vjp", "vjp_launch4", "vjp_launch", "Width"))),
    "fwd_f64_general9": ("eig3_f64.cuh", "eig3_dmul.cuh", "eig3_stats.cuh", "eig3_tile.cuh",
                         ("eig3_f64.cu", ("k_eigvals", "eig_launch4", "eig_launch", "store_aux",
                                          "invariants_of", "aligned16", "Width"))),
}
# HBM bytes per matrix of the two kernels as launched in the step (algorithmic:
# inputs read once, outputs written once)
KERNEL_BYTES = {"vjp_f64_general9": 72 + 24 + 24 + 72, "fwd_f64_general9": 72 + 24 + 32}
# The oracle's eigenvalue evaluation of a general matrix (Algorithms 1, 2, 4,
# 5, 6 as the paper writes them, one rounded operation each), counted with the
# op-counting scalar type of oracle/opcount.cpp (tests/test_oracle_opcount.py
# pins these numbers): the method's literal arithmetic, before any sharing of
# products or fusing into FMAs.
ORACLE_OPS_EIGVALS_GENERAL9 = {"add": 112, "mul": 248, "div": 9, "neg": 7, "sqrt": 2,
                               "atan2": 1, "cos": 3}
# Nominal FP64 pipe of GB300: 2 fused multiply-adds per SM per clock.
FP64_LANES_PER_SM = 2


def _definitions(text, name):
    """Source text of every definition (not a call) of function or struct
    `name` in `text`, from the start of its paragraph to its closing brace."""
    out = []
    for m in re.finditer(r"\bstruct\s+" + name + r"\s*\{", text):
        depth, e = 0, m.end() - 1
        for e in range(m.end() - 1, len(text)):
            depth += text[e] == "{"
            depth -= text[e] == "}"
            if depth == 0:
                break
        start = text.rfind("\n\n", 0, m.start()) + 2
        out.append(text[start:e + 1])
    for m in re.finditer(r"\b" + name + r"\s*\(", text):
        depth, k = 0, m.end() - 1
        for k in range(m.end() - 1, len(text)):  # the parameter list
            depth += text[k] == "("
            depth -= text[k] == ")"
            if depth == 0:
                break
        j = k + 1
        while j < len(text) and text[j] not in "{;":
            j += 1
        if j >= len(text) or text[j] != "{":
            continue
        start = text.rfind("\n\n", 0, m.start()) + 2
        depth, e = 0, j
        for e in range(j, len(text)):
            depth += text[e] == "{"
            depth -= text[e] == "}"
            if depth == 0:
                break
        out.append(text[start:e + 1])
    return out


def kernel_source_md5(sources):
    """Hash of the kernel's source: whole files, or (file, function names) for
    just those functions' definitions in a file that also holds other kernels."""
    import hashlib
    d = os.path.join(ROOT, "paper_2511_00292_gb300", "csrc")
    h = hashlib.md5()
    for src in sources:
        name, funcs = (src, None) if isinstance(src, str) else src
        with open(os.path.join(d, name), "r") as f:
            text = f.read()
        if funcs is None:
            h.update(text.encode())
        else:
            for fn in funcs:
                defs = _definitions(text, fn)
                if not defs:
                    raise ValueError(f"{fn} not defined in {name}")
                h.update("".join(defs).encode())
    return h.hexdigest()


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's shard: every rank processes its own matrices."""
    return base + 7919 * rank


def max_over_ranks(value: float, device) -> float:
    """Max of a per-rank timing over the process group (identity without one)."""
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world: int, per_rank_units: int, ms: float) -> float:
    """Whole-job throughput in G units/s from the max-over-ranks step time."""
    return world * per_rank_units / (ms * 1e-3) / 1e9


def e2e_shift(world: int, per_rank_bytes: float, available: float) -> int:
    """Halvings of each rank's end-to-end batch so that the page-locked host
    buffers of all ranks (they share the node's memory) stay within 70 % of
    the available host memory; at most 6 (1/64 of the batch)."""
    shift = 0
    while shift < 6 and world * per_rank_bytes / (1 << shift) > 0.7 * available:
        shift += 1
    return shift


def host_available_bytes() -> float:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return float(line.split()[1]) * 1024
    except OSError:
        pass
    return float("inf")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def timed(fn, steps, stream):
    """Average milliseconds of fn() over `steps` runs, CUDA events on `stream`."""
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(steps):
        fn()
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e) / steps


# --------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle on the host cores
# --------------------------------------------------------------------------

def oracle_step(oracle, S64, G64, wS, wG, threads):
    """One forward + backward of the oracle over (S64 symmetric, G64 general),
    chunked over `threads` host threads (the C calls release the GIL).
    Returns the eigenvalues of both halves."""
    def chunks(n):
        k = max(1, threads)
        return [(n * i // k, n * (i + 1) // k) for i in range(k)]

    lamS = np.empty((S64.shape[0], 3))
    lamG = np.empty((G64.shape[0], 3))

    def work(args):
        X, w, layout, lo, hi, out = args
        out[lo:hi] = oracle.eigvals(X[lo:hi], layout=layout)
        oracle.eigvals_grad(X[lo:hi], w[lo:hi], layout=layout)

    jobs = [(S64, wS, oracle.SYM6, lo, hi, lamS) for lo, hi in chunks(S64.shape[0])]
    jobs += [(G64, wG, oracle.GENERAL9, lo, hi, lamG) for lo, hi in chunks(G64.shape[0])]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(work, jobs))
    return lamS, lamG


def oracle_sample(n_half, seed, device="cpu"):
    import workloads as W
    w5 = W.workload5(n=2 * n_half, device=device, seed=seed)
    S, G = w5["sym6"], w5["general9"]
    return (S.A.double().cpu().numpy(), G.A.cpu().numpy(), S.extra["w"].double().cpu().numpy(),
            G.extra["w"].cpu().numpy())


def run_reference(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    n_half = 1 << 21
    S64, G64, wS, wG = oracle_sample(n_half, seed=4005)
    for _ in range(args.warmup):
        oracle_step(oracle, S64, G64, wS, wG, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(oracle, S64, G64, wS, wG, threads)
    dt = (time.perf_counter() - t0) / args.steps
    value = 2 * n_half / dt / 1e9
    sample = (f"{2 * n_half} matrices per step ({n_half} symmetric FP32-valued + {n_half} general "
              f"FP64) of the mixed workload, eigenvalues + eigenvector-form gradient")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample_matrices_per_step": 2 * n_half},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# --------------------------------------------------------------------------
# Our arm
# --------------------------------------------------------------------------

def measure_fp_peaks(dev, stream):
    """Throughput of the binary64 and binary32 FMA pipes, measured here with the
    loop kernels of libeig3_peaks.so: DFMA chains alone and between integer or
    binary32 work (kinds 0, 4, 5), FFMA chains (kind 3), each over a few chain
    counts and blocks per SM, about 30 ms per launch after a calibration
    launch; the fastest of each pipe is its measured peak."""
    import ctypes
    from paper_2511_00292_gb300 import build as _b
    lib = ctypes.CDLL(_b.PEAKS_LIB)
    lib.eig3_peak_loop.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p, ctypes.c_void_p]
    lib.eig3_peak_loop.restype = ctypes.c_int
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sp = ctypes.c_void_p(stream.cuda_stream)
    runs = []

    def one(kind, chains, bps, thr, target_ms):
        blocks = sms * bps
        out = torch.empty(blocks * thr, dtype=torch.float64 if kind != 3 else torch.float32,
                          device=dev)
        op = ctypes.c_void_p(out.data_ptr())
        iters = 64
        for _ in range(2):
            st = lib.eig3_peak_loop(kind, chains, blocks, thr, iters, op, sp)
            if st != 0:
                raise RuntimeError(f"eig3_peak_loop failed with CUDA error {st}")
        ms = timed(lambda: lib.eig3_peak_loop(kind, chains, blocks, thr, iters, op, sp), 1, stream)
        iters = max(64, int(iters * target_ms / max(ms, 1e-3)))
        ms = timed(lambda: lib.eig3_peak_loop(kind, chains, blocks, thr, iters, op, sp), 1, stream)
        rate = blocks * thr * iters * chains / (ms * 1e-3) / 1e12
        runs.append({"kind": kind, "chains": chains, "blocks_per_sm": bps, "threads": thr,
                     "ms": ms, "T_inst_per_s": rate})
        return rate

    with ClockSampler(dev.index or 0) as clocks:
        fp64 = max(one(kind, c, b, 256, 30.0) for kind in (0, 4, 5) for c in (2, 8)
                   for b in (1, 4))
        fp32 = max(one(3, c, b, 256, 30.0) for c in (8, 16) for b in (4, 8))
        emul = max(one(8, c, b, 256, 30.0) for c in (4, 8) for b in (2, 4))
    return {"fp64_tinst_per_s": fp64, "fp64_tflops_measured": 2.0 * fp64,
            "fp32_tinst_per_s": fp32, "fp32_tflops_measured": 2.0 * fp32,
            "int_dmul_tops_measured": emul,
            "fp64_loops": "DFMA chains alone and between integer or FFMA work, "
                          "2 or 8 chains per thread, 1 or 4 blocks of 256 per SM; best",
            "int_dmul_loops": "binary64 multiplications on the integer pipes (the kernels' "
                              "dmul), 4 or 8 chains per thread, 2 or 4 blocks of 256 per SM; "
                              "best",
            "clocks": clocks.summary(), "runs": runs}


def kernel_roofline(name, label, n, ms, fp, sm_mhz, sms, hbm_gbs):
    """Roofline object of one binary64 kernel launch on the flop basis: its
    binary64 operations per matrix (FMA = 2), those on the FP64 pipe from its
    ncu counters plus the multiplications it forms on the integer pipes
    (dmul, counted from its source), against the two measured peaks added:
    the DFMA loop's flop rate and the integer-pipe multiplication loop's rate.
    Beside it: the same against the FP64 pipe's peak alone, the FP64-pipe
    issue view and the nominal unit-count peak.  Null where the counters are
    stale."""
    c = KERNEL_COUNTERS[name]
    fresh = c["source_md5"] is not None and kernel_source_md5(KERNEL_SOURCES[name]) == c[
        "source_md5"]
    t = ms * 1e-3
    nominal_inst = sms * FP64_LANES_PER_SM * sm_mhz * 1e6 / 1e12         # T inst/s
    peak = fp["fp64_tflops_measured"] + fp["int_dmul_tops_measured"]
    out = {"kernel": label, "bound": "alu", "unit": "TFLOP/s", "counters_fresh": fresh,
           "peak": peak,
           "peak_source": f"measured in this run (libeig3_peaks): fastest DFMA loop, "
                          f"{fp['fp64_tinst_per_s']:.4f} T DFMA/s x 2 flop, plus fastest "
                          f"integer-pipe multiplication loop, "
                          f"{fp['int_dmul_tops_measured']:.4f} T/s",
           "peak_nominal": 2.0 * nominal_inst,
           "peak_nominal_source": f"FP64 pipe alone: {sms} SMs x {FP64_LANES_PER_SM} FP64 FMA "
                                  f"lanes x {sm_mhz:.0f} MHz x 2 flop",
           "fp64_tflops_measured": fp["fp64_tflops_measured"],
           "int_dmul_tops_measured": fp["int_dmul_tops_measured"],
           "fp32_tflops_measured": fp["fp32_tflops_measured"],
           "ms": ms, "matrices": n, "G_matrices_per_s": n / t / 1e9}
    hbm = KERNEL_BYTES[name]
    out["hbm_view"] = {"bytes_per_matrix": hbm, "achieved_gbs": hbm * n / t / 1e9,
                       "peak_gbs": hbm_gbs, "frac": hbm * n / t / 1e9 / hbm_gbs}
    if not fresh:
        out.update(achieved=None, frac=None, frac_vs_fp64_peak=None, frac_vs_nominal=None,
                   frac_issue=None, traffic=None)
        return out
    pipe_flop = 2 * c["dfma"] + c["dmul"] + c["dadd"]
    flop = pipe_flop + c["int_dmul"]
    achieved = flop * n / t / 1e12
    inst_rate = c["fp64_warp_inst_x32"] * n / t / 1e12      # pipe occupancy
    out.update(achieved=achieved, frac=achieved / peak,
               frac_vs_fp64_peak=achieved / fp["fp64_tflops_measured"],
               frac_vs_nominal=achieved / (2.0 * nominal_inst),
               frac_issue=inst_rate / nominal_inst,
               frac_issue_vs_measured_loop=inst_rate / fp["fp64_tinst_per_s"],
               traffic=c["dram_bytes"] * n,
               algorithmic_per_matrix={"flop": flop, "fp64_pipe_inst": c["fp64_pipe_inst"],
                                       "fp64_warp_inst_x32": c["fp64_warp_inst_x32"],
                                       "dfma": c["dfma"], "dmul": c["dmul"], "dadd": c["dadd"],
                                       "int_dmul": c["int_dmul"], "hbm_bytes": hbm},
               mix_ceiling=pipe_flop / (2.0 * c["fp64_warp_inst_x32"]))
    return out


def self_launch_command(gpus: int, argv) -> list:
    """The torchrun command that `bench.py --gpus N` (N > 1, outside torchrun)
    re-executes itself under: one rank per GPU of this node, rendezvous on
    127.0.0.1 at a free port."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
            f"--nproc-per-node={gpus}", "--master-addr=127.0.0.1", f"--master-port={port}",
            os.path.abspath(__file__), *argv]


def run_ours(args):
    import paper_2511_00292_gb300 as eig3
    from paper_2511_00292_gb300 import build as _b
    import workloads as W

    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _b.build()
    eig3.load()
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize(dev)

    # ---- the mixed workload (inputs resident in HBM) ----
    w5 = W.workload5(n=N_MIXED, device=dev, seed=rank_seed(1005, rank))
    S, G = w5["sym6"], w5["general9"]
    nS, nG = S.n, G.n
    lamS = torch.empty(nS, 3, dtype=torch.float32, device=dev)
    gS = torch.empty_like(S.A)
    lamG = torch.empty(nG, 3, dtype=torch.float64, device=dev)
    gG = torch.empty_like(G.A)
    wS, wG = S.extra["w"], G.extra["w"]
    stats = eig3.Stats(dev)

    # One step: eigenvalues and the gradient of sum(w * lambda) for both halves,
    # each in one fused launch (eig3_eigvals_vjp).  The binary64 kernel keeps the
    # FP64 pipe busy with little else; the compensated binary32 kernel uses the
    # FP32 pipes, so it runs on a second stream beside it.
    def vjp_S():
        eig3.eigvals_vjp(S.A, wS, precision="f32c", out=lamS, grad_out=gS, stats=stats)

    def vjp_G():
        eig3.eigvals_vjp(G.A, wG, precision="f64", out=lamG, grad_out=gG, stats=stats)

    s64, s32 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def step():
        s64.wait_stream(stream)
        s32.wait_stream(stream)
        with torch.cuda.stream(s64):
            vjp_G()
        with torch.cuda.stream(s32):
            vjp_S()
        stream.wait_stream(s64)
        stream.wait_stream(s32)

    launches_per_step = 2
    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize(dev)
    stats.reset()

    # ---- timed region: K steps ----
    barrier()
    with ClockSampler(local) as clocks:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
    barrier()
    ms = max_over_ranks(ms, dev)
    value = weak_scaling_value(world, N_MIXED, ms)
    step_stats = stats.read()

    # ---- per-kernel durations (each launch alone, events on the launch stream) ----
    lamG4 = torch.empty(nG, 4, dtype=torch.float64, device=dev)

    def fwd_G():
        eig3.eigvals(G.A, precision="f64", return_aux=True, out=lamG, aux_out=lamG4, stats=stats)

    kern = {}
    for name, fn in (("vjp_f32c_sym6", vjp_S), ("vjp_f64_general9", vjp_G),
                     ("fwd_f64_general9", fwd_G)):
        fn()
        kern[name] = timed(fn, args.steps, stream)
    del lamG4
    fp = measure_fp_peaks(dev, stream)
    pk, pk_src = peaks()
    sm_mhz = clocks.summary().get("sm_mhz") or float(pk.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    hbm = float(pk.get("hbm_gbs", 6800.0))
    roofline = kernel_roofline(
        "vjp_f64_general9", "k_eigvals_vjp<general9, f64> (fused forward + vector-Jacobian "
        "product, binary64; the step's dominant launch, 2^27 matrices)", nG,
        kern["vjp_f64_general9"], fp, sm_mhz, sms, hbm)
    roofline["hbm_view"]["peak_source"] = pk_src
    roofline["kernel_ms"] = kern
    roofline_fwd = kernel_roofline(
        "fwd_f64_general9", "k_eigvals<general9, f64, aux, stats> (binary64 forward, "
        "2^27 matrices)", nG, kern["fwd_f64_general9"], fp, sm_mhz, sms, hbm)
    ops = ORACLE_OPS_EIGVALS_GENERAL9
    lit = ops["add"] + ops["mul"] + ops["div"]
    roofline_fwd["oracle_literal_ops_per_matrix"] = dict(ops, flop=lit)
    roofline_fwd["frac_oracle_literal_flop"] = lit * nG / (kern["fwd_f64_general9"] * 1e-3) / 1e12 \
        / roofline_fwd["peak"]

    # ---- the other workloads' paths (fwd, fwd+bwd, FP64 vs compensated FP32) ----
    paths = {}
    if not args.skip_paths:
        paths = measure_paths(eig3, W, dev, stream, args.steps, S=S, G=G, step_fns=dict(
            vjp_S=vjp_S, vjp_G=vjp_G, s64=s64, s32=s32), lam=(lamS, lamG), grad=(gS, gG))

    # ---- end to end through host buffers (pinned), public API ----
    e2e = None
    if not args.skip_e2e:
        per_rank = (S.A.numel() * 4 + nS * 12) * 2 + (G.A.numel() * 8 + nG * 24) * 2 + (1 << 30)
        shift = e2e_shift(world, per_rank, host_available_bytes())
        barrier()
        e2e = measure_e2e(eig3, S, G, dev, stream, args.steps, shift)
        if dist:  # whole job: every rank streamed its own batch; the slowest sets the time
            e2e["ms_per_step"] = max_over_ranks(e2e["ms_per_step"], dev)
            e2e["value"] = weak_scaling_value(world, e2e["matrices_per_gpu"], e2e["ms_per_step"])
            e2e["h2d_bytes_per_step"] *= world
            e2e["d2h_bytes_per_step"] *= world

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64+f32c", "data": "synthetic",
           "config": {"workload": WORKLOAD, "matrices_per_gpu": N_MIXED,
                      "l2": "inputs ~18 GB/step > 129 MB L2, no flush needed",
                      "launch": "2 kernels per step (eig3_eigvals_vjp for each half), the "
                                "binary32 one on a second stream beside the binary64 one"},
           "roofline": roofline, "roofline_fwd": roofline_fwd, "fp_peaks": fp,
           "gpu_launches": launches_per_step * args.steps,
           "clocks": clocks.summary(), "e2e": e2e, "paths": paths, "stats": step_stats}

    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only) ----
    if rank == 0 and world == 1 and not args.skip_cpu:
        out["cpu_baseline"], out["max_err_over_bound"], out["err_vs_exact"] = cpu_baseline(
            eig3, W, dev, S, G, lamS, lamG)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        tdist.destroy_process_group()
    return 0


def measure_paths(eig3, W, dev, stream, steps, S, G, step_fns, lam, grad):
    paths = {}
    steps = max(steps, 3)
    vjp_S, vjp_G, s64, s32 = (step_fns[k] for k in ("vjp_S", "vjp_G", "s64", "s32"))

    def step_on(base):
        s64.wait_stream(base)
        s32.wait_stream(base)
        with torch.cuda.stream(s64):
            vjp_G()
        with torch.cuda.stream(s32):
            vjp_S()
        base.wait_stream(s64)
        base.wait_stream(s32)

    # the benchmark step in the literal form of workload 5: 10 forward + backward
    # steps captured once as one CUDA graph and replayed
    step_on(stream)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cap = torch.cuda.current_stream(dev)
        for _ in range(10):
            step_on(cap)
    graph.replay()
    torch.cuda.synchronize(dev)
    reps = max(1, steps // 10 + 1)
    tg = timed(graph.replay, reps, stream) / 10
    paths["mixed_step_graph_10_steps"] = {
        "ms_per_step": tg, "G_matrices_per_s": (S.n + G.n) / tg / 1e6,
        "form": "10 fused fwd+bwd steps captured once in a CUDA graph (20 kernel nodes on two "
                "streams), replayed"}
    del graph
    # the same step unfused (eig3_eigvals with adjoint inputs, then
    # eig3_eigvals_backward, for each half), as the autograd path runs it
    lamS, lamG = lam
    gS, gG = grad
    auxS = torch.empty(S.n, 4, dtype=torch.float32, device=dev)
    auxG = torch.empty(G.n, 4, dtype=torch.float64, device=dev)
    wS, wG = S.extra["w"], G.extra["w"]

    def unfused():
        s64.wait_stream(stream)
        s32.wait_stream(stream)
        with torch.cuda.stream(s64):
            eig3.eigvals(G.A, return_aux=True, out=lamG, aux_out=auxG)
            eig3.eigvals_backward(G.A, wG, aux=auxG, out=gG)
        with torch.cuda.stream(s32):
            eig3.eigvals(S.A, precision="f32c", return_aux=True, out=lamS, aux_out=auxS)
            eig3.eigvals_backward(S.A, wS, aux=auxS, precision="f32c", out=gS)
        stream.wait_stream(s64)
        stream.wait_stream(s32)

    unfused()
    tu = timed(unfused, steps, stream)
    paths["mixed_step_unfused"] = {"ms_per_step": tu, "G_matrices_per_s": (S.n + G.n) / tu / 1e6,
                                   "form": "eig3_eigvals + eig3_eigvals_backward per half, "
                                           "4 launches on two streams"}
    del auxS, auxG
    torch.cuda.empty_cache()
    b2 = W.workload2(n=1 << 26, device=dev)
    lam = torch.empty(b2.n, 3, dtype=torch.float64, device=dev)
    t = timed(lambda: eig3.eigvals(b2.A, out=lam), steps, stream)
    paths["fwd_f64_general9_2^26"] = {"G_matrices_per_s": b2.n / t / 1e6, "ms": t}
    del b2, lam
    b3 = W.workload3(n=1 << 27, device=dev)
    l3 = torch.empty(b3.n, 3, dtype=torch.float32, device=dev)
    tc = timed(lambda: eig3.eigvals(b3.A, precision="f32c", out=l3), steps, stream)
    td = timed(lambda: eig3.eigvals(b3.A, precision="f64", out=l3), steps, stream)
    ta = timed(lambda: eig3.eigvals(b3.A, precision="f32c64", out=l3), steps, stream)
    paths["fwd_sym6_fp32_storage_2^27"] = {
        "f32c_G_matrices_per_s": b3.n / tc / 1e6, "f64_G_matrices_per_s": b3.n / td / 1e6,
        "f32c_speedup_over_f64": td / tc,
        "f32c64_G_matrices_per_s": b3.n / ta / 1e6}
    del b3, l3
    b4 = W.workload4(n=1 << 24, device=dev)
    lam4 = torch.empty(b4.n, 3, dtype=torch.float64, device=dev)
    aux4 = torch.empty(b4.n, 4, dtype=torch.float64, device=dev)
    g4 = torch.empty_like(b4.A)
    w4 = b4.extra["w"]

    def fb():
        eig3.eigvals(b4.A, out=lam4, return_aux=True, aux_out=aux4)
        eig3.eigvals_backward(b4.A, w4, aux=aux4, out=g4)

    t4 = timed(fb, steps, stream)
    paths["fwd_bwd_f64_general9_2^24"] = {"G_matrices_per_s": b4.n / t4 / 1e6, "ms": t4}
    t4v = timed(lambda: eig3.eigvals_vjp(b4.A, w4, out=lam4, grad_out=g4), steps, stream)
    paths["vjp_f64_general9_2^24"] = {"G_matrices_per_s": b4.n / t4v / 1e6, "ms": t4v}
    P4 = torch.empty(b4.n, 27, dtype=torch.float64, device=dev)
    tp = timed(lambda: eig3.eigprojectors(b4.A, out=P4, return_eigvals=True, lam_out=lam4),
               steps, stream)
    paths["eigprojectors_f64_general9_2^24"] = {"G_matrices_per_s": b4.n / tp / 1e6, "ms": tp}
    del b4, lam4, aux4, g4, P4
    b3 = W.workload3(n=1 << 25, device=dev)
    P3 = torch.empty(b3.n, 27, dtype=torch.float32, device=dev)
    tq = timed(lambda: eig3.eigprojectors(b3.A, precision="f32c", out=P3), steps, stream)
    paths["eigprojectors_f32c_sym6_2^25"] = {"G_matrices_per_s": b3.n / tq / 1e6, "ms": tq}
    del b3, P3
    # the paper's comparison variants at scale: time, and distance from the
    # method's eigenvalues in units of its first-order bound, per spectrum kind
    b2 = W.workload2(n=1 << 24, device=dev, seed=1102)
    lv = torch.empty(b2.n, 3, dtype=torch.float64, device=dev)
    lp = torch.empty_like(lv)
    bound = b2.kappa * torch.linalg.vector_norm(b2.A, dim=1) * 2.0 ** -53
    kinds = b2.extra["kinds"]
    var = {}
    for v in ("present", "naive", "naive_tensor"):
        out = lp if v == "present" else lv
        tv = timed(lambda: eig3.eigvals_variant(b2.A, v, invariants=False, lam_out=out), steps,
                   stream)
        var[v] = {"G_matrices_per_s": b2.n / tv / 1e6}
        if v != "present":
            r = torch.nan_to_num((lv - lp).abs().amax(dim=1) / bound, nan=float("inf"))
            for k, name in ((0, "distinct"), (1, "near_double"), (2, "near_triple")):
                rk = r[kinds == k]
                var[v][name] = {"max_dist_over_bound": float(rk.amax()),
                                "frac_beyond_16_bounds": float((rk > 16).float().mean())}
    paths["variants_f64_general9_2^24"] = var
    del b2, lv, lp, bound, kinds
    # the guarded binary64 precision: cost on well-conditioned general matrices
    # (workload 2) and on ill-conditioned ones (kappa up to 1e4), with the
    # share of matrices the guard switched to the QR algorithm
    guard = {}
    for name, bt in (("workload2_2^24", W.workload2(n=1 << 24, device=dev, seed=1103)),
                     ("ill_conditioned_kappa_le_1e4_2^24",
                      W.illconditioned(1 << 24, dev, seed=1104, log10_kappa_max=4.0))):
        lg = torch.empty(bt.n, 3, dtype=torch.float64, device=dev)
        lpl = torch.empty_like(lg)
        st = eig3.Stats(dev)
        tg = timed(lambda: eig3.eigvals(bt.A, precision="f64g", out=lg), steps, stream)
        tp = timed(lambda: eig3.eigvals(bt.A, out=lpl), steps, stream)
        eig3.eigvals(bt.A, precision="f64g", out=lg, stats=st)
        guard[name] = {"f64g_G_matrices_per_s": bt.n / tg / 1e6,
                       "f64_G_matrices_per_s": bt.n / tp / 1e6,
                       "switched_fraction": st.read()["n_guarded"] / bt.n}
        del bt, lg, lpl
    paths["guarded_f64_general9"] = guard
    # Mohr-Coulomb yield value + gradient (Section "Application"), fused
    sf = W.stress_field(1 << 25, dev, seed=1006)
    f5 = torch.empty(sf.n, dtype=torch.float64, device=dev)
    g5 = torch.empty_like(sf.A)
    tm = timed(lambda: eig3.mohr_coulomb(sf.A, grad=True, out=f5, grad_out=g5), steps, stream)
    paths["mohr_coulomb_f64_sym6_2^25"] = {"G_matrices_per_s": sf.n / tm / 1e6, "ms": tm}
    A32 = sf.A.float()
    del sf, f5, g5
    f6 = torch.empty(A32.shape[0], dtype=torch.float32, device=dev)
    g6 = torch.empty_like(A32)
    tn = timed(lambda: eig3.mohr_coulomb(A32, precision="f32c", grad=True, out=f6, grad_out=g6),
               steps, stream)
    paths["mohr_coulomb_f32c_sym6_2^25"] = {"G_matrices_per_s": A32.shape[0] / tn / 1e6, "ms": tn}
    del A32, f6, g6
    torch.cuda.empty_cache()
    return paths


def measure_e2e(eig3, S, G, dev, stream, steps, shift=0, chunk=1 << 21):
    """The same step on host-resident data through the public API
    (paper_2511_00292_gb300.host.HostPipeline): the matrices and loss weights
    start in pinned host memory and the eigenvalues and gradients end there;
    every host-to-device and device-to-host copy is inside the timed region,
    overlapped with the kernels chunk by chunk on separate streams.  `shift`
    halves the batch that many times (host memory shared by several ranks)."""
    from paper_2511_00292_gb300.host import (HostPipeline, huge_page_fraction, pinned_copy,
                                             pinned_empty)
    mS, mG = S.n >> shift, G.n >> shift
    hS = pinned_copy(S.A[:mS])
    hG = pinned_copy(G.A[:mG])
    hwS = pinned_copy(S.extra["w"][:mS])
    hwG = pinned_copy(G.extra["w"][:mG])
    olS = pinned_empty((mS, 3), torch.float32)
    olG = pinned_empty((mG, 3), torch.float64)
    ogS = pinned_empty(hS.shape, hS.dtype)
    ogG = pinned_empty(hG.shape, hG.dtype)
    # Some host buffers copy at a few GB/s for their whole life (measured: 3.8 to
    # 10 GB/s against 211 for the others, with or without huge pages, on a single
    # NUMA node), and one such buffer holds the streamed step at 140-520 ms
    # instead of 107.  Each buffer's own copy is timed here, untimed setup, and
    # a buffer below 140 GB/s is made again (up to three times).
    big = max(t.numel() * t.element_size() for t in (hS, hG, hwS, hwG, olS, olG, ogS, ogG))
    scratch = torch.empty(big, dtype=torch.uint8, device=dev)
    rates, remade = {}, []

    def copy_gbs(t, to_dev):
        nb = t.numel() * t.element_size()
        h = t.view(-1).view(torch.uint8)
        if to_dev:
            fn = lambda: scratch[:nb].copy_(h, non_blocking=True)
        else:
            fn = lambda: h.copy_(scratch[:nb], non_blocking=True)
        return nb / (timed(fn, 1, stream) * 1e-3) / 1e9

    def checked(name, t, fill):
        to_dev = fill is not None
        for attempt in range(4):
            r = copy_gbs(t, to_dev)
            if r >= 140.0 or attempt == 3:
                break
            remade.append(name)
            t = pinned_copy(fill) if to_dev else pinned_empty(t.shape, t.dtype)
        rates[name] = round(r, 1)
        return t

    hS = checked("A_sym6", hS, S.A[:mS])
    hG = checked("A_general9", hG, G.A[:mG])
    hwS = checked("w_sym6", hwS, S.extra["w"][:mS])
    hwG = checked("w_general9", hwG, G.extra["w"][:mG])
    olS, olG = checked("lam_sym6", olS, None), checked("lam_general9", olG, None)
    ogS, ogG = checked("grad_sym6", ogS, None), checked("grad_general9", ogG, None)
    del scratch
    huge = min(huge_page_fraction(t) for t in (hS, hG, hwS, hwG, olS, olG, ogS, ogG))
    h2d = sum(t.numel() * t.element_size() for t in (hS, hG, hwS, hwG))
    d2h = sum(t.numel() * t.element_size() for t in (olS, olG, ogS, ogG))
    pipe = HostPipeline(dev, chunk=chunk, depth=3)

    graph = pipe.capture([(hS, hwS, olS, ogS, None, "f32c"), (hG, hwG, olG, ogG, None, "f64")])

    def step():
        graph.replay()

    step()
    torch.cuda.synchronize(dev)
    k = max(1, steps)
    ms = timed(step, k, stream)
    # the copy ceiling on this machine: the same pinned buffers, 1 GiB each way
    # at once (host-to-device on one stream, device-to-host on another)
    nb = 1 << 30
    src_h = hG.view(-1).view(torch.uint8)[:nb]
    dst_h = pinned_empty(nb, torch.uint8)
    dbuf = torch.empty(2, nb, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def both():
        s1.wait_stream(stream)
        s2.wait_stream(stream)
        with torch.cuda.stream(s1):
            dbuf[0].copy_(src_h, non_blocking=True)
        with torch.cuda.stream(s2):
            dst_h.copy_(dbuf[1], non_blocking=True)
        stream.wait_stream(s1)
        stream.wait_stream(s2)

    both()
    t_both = timed(both, 3, stream) * 1e-3
    each_gbs = nb / t_both / 1e9
    floor_ms = max(h2d, d2h) / (each_gbs * 1e9) * 1e3
    del dbuf, dst_h
    # the results are the device results: spot-check one chunk of each half
    ok = bool(torch.equal(olG[:1024], eig3.eigvals(G.A[:1024]).cpu())) and \
        bool(torch.equal(olS[:1024], eig3.eigvals(S.A[:1024], precision="f32c").cpu()))
    # the same step with the C entry point given the host buffers themselves
    # (eig3_eigvals_vjp on page-locked host pointers: the kernels read A and w
    # and write lambda and the gradient over NVLink-C2C, no copies), for
    # comparison with the copy-engine pipeline above
    s32 = torch.cuda.Stream(dev)

    def zero_copy():
        s32.wait_stream(stream)
        eig3.eigvals_vjp(hG, hwG, precision="f64", out=olG, grad_out=ogG, device=dev)
        with torch.cuda.stream(s32):
            eig3.eigvals_vjp(hS, hwS, precision="f32c", out=olS, grad_out=ogS, device=dev)
        stream.wait_stream(s32)

    zero_copy()
    torch.cuda.synchronize(dev)
    zms = timed(zero_copy, 2, stream)
    zok = bool(torch.equal(olG[:1024], eig3.eigvals(G.A[:1024]).cpu()))
    del hS, hG, hwS, hwG, olS, olG, ogS, ogG, pipe
    return {"value": (mS + mG) / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "matrices_per_gpu": mS + mG,
            "mode": "pinned host buffers (host.pinned_empty: huge-page mappings registered "
                    f"with CUDA), chunks of 2^{chunk.bit_length() - 1} streamed through 3 device slots "
                    "(H2D / kernels / D2H on 3 streams), captured once as a CUDA graph",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": k,
            "host_huge_page_fraction_min": huge, "host_buffers_remade": remade,
            "host_buffer_copy_gbs": rates,
            "results_match_device": ok,
            "copy_roofline": {"both_directions_gbs_each": each_gbs, "floor_ms": floor_ms,
                              "frac": floor_ms / ms},
            "zero_copy": {"value": (mS + mG) / (zms * 1e-3) / 1e9, "unit": UNIT,
                          "ms_per_step": zms, "steps": 2, "results_match_device": zok,
                          "mode": "eig3_eigvals_vjp on the page-locked host buffers "
                                  "themselves (kernels read and write host memory over "
                                  "NVLink-C2C), the binary32 half on a second stream"}}


def ratio_stats(err, bound):
    """max and p99.9 of err / bound over the finite rows (0/0 counts as 0)."""
    err = np.asarray(err, dtype=np.float64)
    bound = np.asarray(bound, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(err == 0, 0.0, err / bound)
    r = r[np.isfinite(err)]
    if r.size == 0:
        return {"max": None, "p999": None}
    return {"max": float(np.max(r)), "p999": float(np.quantile(r, 0.999))}


def err_vs_exact(eig3, W, dev, S, G, lamS, lamG, k=1 << 13):
    """Distance of the GPU results from the exact values of the stored matrices
    (oracle.eigvals_exact / invariants_exact, rational and 60-digit
    arithmetic), per eigenvalue and per invariant, in units of the paper's
    first-order bounds at C = 1 (Lemma of Section "Eigenvalues": kappa
    ||A||_F u; Sections I1, J2, J3, Delta for the invariants), with u = 2^-53
    for the binary64 path and 2^-24 for the compensated binary32 one.
    Samples of k matrices per workload (all 4160 of workload 1), both halves
    of the benchmark step from the step's own eigenvalues."""
    import oracle
    procs = os.cpu_count() or 1
    U64, U32 = 2.0 ** -53, 2.0 ** -24
    sets = []
    A1 = W.workload1("cpu")["general9"].A
    d1 = A1.to(dev)
    sets.append(("workload1_general9_f64", A1.numpy(), 0, np.ones(A1.shape[0]), eig3.eigvals(d1),
                 eig3.invariants(d1), U64))
    b2 = W.workload2(n=k, device="cpu", seed=1202)
    d2 = b2.A.to(dev)
    sets.append(("workload2_general9_f64", b2.A.numpy(), 0, b2.kappa.numpy(), eig3.eigvals(d2),
                 eig3.invariants(d2), U64))
    b3 = W.workload3(n=k, device="cpu", seed=1203)
    d3 = b3.A.to(dev)
    sets.append(("workload3_sym6_f32c", b3.A.double().numpy(), 1, np.ones(k),
                 eig3.eigvals(d3, precision="f32c"), eig3.invariants(d3, precision="f32c"), U32))
    b4 = W.workload4(n=k, device="cpu", seed=1204)
    d4 = b4.A.to(dev)
    lam4, _ = eig3.eigvals_vjp(d4, b4.extra["w"].to(dev))
    sets.append(("workload4_general9_f64_vjp", b4.A.numpy(), 0, b4.kappa.numpy(), lam4,
                 eig3.invariants(d4), U64))
    iS = torch.as_tensor(W.sample_indices(S.n, k, seed=13), device=S.A.device)
    iG = torch.as_tensor(W.sample_indices(G.n, k, seed=14), device=G.A.device)
    sets.append(("workload5_sym6_f32c_half", S.A[iS].double().cpu().numpy(), 1, np.ones(k),
                 lamS[iS], eig3.invariants(S.A[iS].contiguous(), precision="f32c"), U32))
    sets.append(("workload5_general9_f64_half", G.A[iG].cpu().numpy(), 0, G.kappa[iG].cpu().numpy(),
                 lamG[iG], eig3.invariants(G.A[iG].contiguous()), U64))
    out = {"bound": "C = 1: kappa ||A||_F u for eigenvalues, the first-order bounds of Sections "
                    "I1, J2, J3, Delta for the invariants; exact values of the stored matrices",
           "sets": {}}
    t0 = time.perf_counter()
    for name, A, lay, kappa, lam, inv, u in sets:
        lam_x = oracle.map_eigvals_exact(A, lay, procs)
        inv_x = oracle.map_invariants_exact(A, lay, procs)
        b = oracle.bounds(A, kappa, layout=lay, u=u)
        lam_g = lam.double().cpu().numpy()
        inv_g = inv.cpu().numpy()
        real = np.all(np.isfinite(lam_x), axis=1)       # complex spectra of fl(A) are NaN
        e = {"matrices": int(A.shape[0]), "real_spectra": int(real.sum())}
        for j in range(3):
            e[f"lambda{j + 1}"] = ratio_stats(np.abs(lam_g[real, j] - lam_x[real, j]),
                                              b[real, 4])
        # the compensated invariants are claimed at u32^2: their bounds at that u
        bi = b if u == U64 else oracle.bounds(A, kappa, layout=lay, u=u * u)
        e["invariant_bound_u"] = "2^-53" if u == U64 else "2^-48"
        for j, nm in enumerate(("I1", "J2", "J3", "Delta")):
            e[nm] = ratio_stats(np.abs(inv_g[:, j] - inv_x[:, j]), bi[:, j])
        out["sets"][name] = e
    out["cpu_seconds"] = time.perf_counter() - t0
    out["processes"] = procs
    return out


def cpu_baseline(eig3, W, dev, S, G, lamS, lamG):
    """The FP64 oracle (as it stands) on the host cores, on a bounded sample of
    the workload; the same sample gives the max error over the stability bound
    of the GPU results against the oracle.  Also workload 1 timed whole (the
    oracle's forward in ms) and the distance of the GPU results from the exact
    eigenvalues and invariants (err_vs_exact)."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    k = 1 << 24  # 2 x 2^24 matrices: about 12 s of CPU time on 16 Grace cores
    iS = torch.as_tensor(W.sample_indices(S.n, k, seed=11), device=S.A.device)
    iG = torch.as_tensor(W.sample_indices(G.n, k, seed=12), device=G.A.device)
    S64 = S.A[iS].double().cpu().numpy()
    G64 = G.A[iG].cpu().numpy()
    wS = S.extra["w"][iS].double().cpu().numpy()
    wG = G.extra["w"][iG].cpu().numpy()
    t0 = time.perf_counter()
    refS, refG = oracle_step(oracle, S64, G64, wS, wG, threads)
    dt = time.perf_counter() - t0
    value = (S64.shape[0] + G64.shape[0]) / dt / 1e9
    # one host thread on the first 2^18 + 2^18 matrices of the same sample
    m = 1 << 18
    t1 = time.perf_counter()
    oracle_step(oracle, S64[:m], G64[:m], wS[:m], wG[:m], 1)
    ns_1t = (time.perf_counter() - t1) / (2 * m) * 1e9
    # workload 1 whole (4096 + 64 symmetric matrices, general 9-entry storage):
    # the oracle's forward, one thread and all threads, best of 3
    A1 = W.workload1("cpu")["general9"].A.numpy()
    t_1, t_all = [], []
    for _ in range(3):
        t = time.perf_counter()
        oracle.eigvals(A1)
        t_1.append(time.perf_counter() - t)
        t = time.perf_counter()
        oracle.eigvals_mt(A1, nthreads=threads)
        t_all.append(time.perf_counter() - t)
    # accuracy of the GPU results on this sample, against the oracle
    refS = np.sort(refS, axis=1)
    refG = np.sort(refG, axis=1)
    bS = oracle.bounds(S64, 1.0, layout=oracle.SYM6, u=2.0 ** -24)[:, 4]
    bG = oracle.bounds(G64, G.kappa[iG].cpu().numpy())[:, 4]
    eS = np.abs(lamS[iS].double().cpu().numpy() - refS).max(axis=1)
    eG = np.abs(lamG[iG].cpu().numpy() - refG).max(axis=1)
    cpu = {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{S64.shape[0]} symmetric + {G64.shape[0]} general matrices of the "
                     f"mixed workload, eigenvalues + eigenvector-form gradient, "
                     f"{dt:.2f} s wall on {threads} threads "
                     f"(about {dt * threads:.0f} s of CPU time)",
           "single_thread_ns_per_matrix": ns_1t,
           "workload1_forward_ms": {"matrices": int(A1.shape[0]), "one_thread": 1e3 * min(t_1),
                                    "all_threads": 1e3 * min(t_all), "threads": threads}}
    err = {"f32c_sym6": float(np.max(eS / bS)), "f64_general9": float(np.max(eG / bG)),
           "f32c_sym6_p999": float(np.quantile(eS / bS, 0.999)),
           "f64_general9_p999": float(np.quantile(eG / bG, 0.999)),
           "bound": "kappa ||A||_F u (u = 2^-24 for f32c, 2^-53 for f64; C = 1), GPU against "
                    "the oracle",
           "sample_matrices": int(S64.shape[0] + G64.shape[0])}
    return cpu, err, err_vs_exact(eig3, W, dev, S, G, lamS, lamG)


KERNELS = ("fwd_f64_general9", "bwd_f64_general9", "fwd_f32c_sym6", "bwd_f32c_sym6",
           "fwd_f64_sym6", "mc_f64_sym6", "mc_f32c_sym6", "guard_f64_illcond",
           "proj_f32c_sym6", "vjp_f64_general9", "vjp_f32c_sym6", "eig_f32c_sym6")


def run_single(args):
    """W + K launches of one library kernel at size n (for profiler captures)."""
    import paper_2511_00292_gb300 as eig3
    from paper_2511_00292_gb300 import build as _b
    import workloads as W
    dev = torch.device("cuda", 0)
    _b.build()
    n = args.n
    if args.only in ("guard_f64_illcond", "proj_f32c_sym6"):
        if args.only == "guard_f64_illcond":
            A = W.illconditioned(n, dev, seed=1104, log10_kappa_max=4.0).A
            lam = torch.empty(n, 3, dtype=torch.float64, device=dev)
            fn = lambda: eig3.eigvals(A, precision="f64g", out=lam)
        else:
            A = W.workload3(n=n, device=dev).A
            P = torch.empty(n, 3, 3, 3, dtype=torch.float32, device=dev)
            fn = lambda: eig3.eigprojectors(A, precision="f32c", out=P)
        for _ in range(args.warmup):
            fn()
        ms = timed(fn, args.steps, torch.cuda.current_stream(dev))
        print(json.dumps({"kernel": args.only, "n": n, "ms": ms, "G_matrices_per_s": n / ms / 1e6}))
        return 0
    if args.only.startswith("mc_"):
        prec = "f32c" if "f32c" in args.only else "f64"
        A = W.stress_field(n, dev, seed=1006).A
        A = A.float() if prec == "f32c" else A
        f = torch.empty(n, dtype=A.dtype, device=dev)
        g = torch.empty_like(A)
        fn = lambda: eig3.mohr_coulomb(A, precision=prec, grad=True, out=f, grad_out=g)
        for _ in range(args.warmup):
            fn()
        ms = timed(fn, args.steps, torch.cuda.current_stream(dev))
        print(json.dumps({"kernel": args.only, "n": n, "ms": ms, "G_matrices_per_s": n / ms / 1e6}))
        return 0
    if "general9" in args.only:
        b = W.workload4(n=n, device=dev)
        A, w = b.A, b.extra["w"]
        prec = "f64"
    else:
        b = W.workload3(n=n, device=dev)
        A, w = b.A, torch.randn(n, 3, dtype=torch.float32, device=dev)
        prec = "f32c" if "f32c" in args.only else "f64"
    lam, aux = eig3.eigvals(A, precision=prec, return_aux=True)
    g = torch.empty_like(A)
    st = eig3.Stats(dev)
    if args.only.startswith("fwd"):
        fn = lambda: eig3.eigvals(A, precision=prec, return_aux=True, out=lam, aux_out=aux,
                                  stats=st)
    elif args.only.startswith("eig"):  # eigenvalues alone (no adjoint inputs, no statistics)
        fn = lambda: eig3.eigvals(A, precision=prec, out=lam)
    elif args.only.startswith("vjp"):
        fn = lambda: eig3.eigvals_vjp(A, w, precision=prec, out=lam, grad_out=g, stats=st)
    else:
        fn = lambda: eig3.eigvals_backward(A, w, aux=aux, precision=prec, out=g)
    for _ in range(args.warmup):
        fn()
    ms = timed(fn, args.steps, torch.cuda.current_stream(dev))
    print(json.dumps({"kernel": args.only, "n": n, "ms": ms, "G_matrices_per_s": n / ms / 1e6}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--skip-paths", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--only", choices=KERNELS, default=None,
                    help="time one kernel alone at size --n (profiler captures)")
    ap.add_argument("--n", type=int, default=1 << 22)
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP64 / FP32 pipe peaks only and print them")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: re-run this command under torchrun
        return subprocess.call(self_launch_command(args.gpus, sys.argv[1:]))
    if args.impl == "reference":
        return run_reference(args)
    if args.peaks:
        from paper_2511_00292_gb300 import build as _b
        _b.build()
        dev = torch.device("cuda", env_int("LOCAL_RANK", 0))
        torch.cuda.set_device(dev)
        fp = measure_fp_peaks(dev, torch.cuda.current_stream(dev))
        print(json.dumps(fp), flush=True)
        return 0
    if args.only:
        return run_single(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
