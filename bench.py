"""Benchmark: batched stable closed-form 3x3 eigenvalues on GB300.

One step = one forward + backward pass of the whole path over the mixed
workload of 2^28 matrices per GPU: 2^27 symmetric 6-entry binary32 matrices
through the compensated binary32 kernels and 2^27 general 9-entry binary64
matrices through the binary64 kernels (invariants I1, J2, J3, Delta ->
triple angle -> eigenvalues -> adjoint), the two halves on two streams.
Inputs are resident in HBM and larger than L2 (about 18 GB per step), so no
L2 flush is needed between steps.

Printed (rank 0, one JSON line): whole-job throughput in G matrices/s, the
roofline of the dominant kernel (binary64 general forward) measured live with
CUDA events, per-path throughputs of the other workloads' shapes, the CPU
oracle timed on the host cores on a bounded sample (with the max error over
the stability bound of the GPU results on that sample), an end-to-end number
through host buffers, and SM clocks sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
            "triple-perturbed, the binary32 half on a second stream")

# Per-matrix counts of the binary64 general 9-entry forward kernel with
# adjoint outputs and statistics (the launch of the timed step), taken with ncu
# on n = 2^22 (bench.py --only fwd_f64_general9): thread-level instructions on
# the FP64 pipe, of which DFMA / DMUL / DADD, and DRAM bytes read + written.
# They describe the kernel source whose hash is recorded here; when the source
# changes they are reported as stale and the traffic as null.
FWD_F64_COUNTERS = {
    "source_md5": "037d9baa6a11164747fac4e74e25d8f1",
    "fp64_pipe_inst": 171.10, "dfma": 84.0, "dmul": 63.0, "dadd": 17.0,
    "dram_bytes": (302.036992e6 + 193.370112e6) / 4194304,
}
# the headers whole, and of eig3_f64.cu the forward kernel and its launchers
FWD_F64_SOURCES = ("eig3_f64.cuh", "eig3_stats.cuh", "eig3_tile.cuh",
                   ("eig3_f64.cu", ("k_eigvals", "eig_launch4", "eig_launch")))
# FP64 pipe of GB300: 2 FMA lanes per SM (measured with a DFMA loop: 0.598 T
# DFMA/s at 1.97 GHz on 152 SMs), so the peak is SMs x 2 x clock instructions/s.
FP64_LANES_PER_SM = 2


def _definitions(text, name):
    """Source text of every definition (not a call) of function `name` in `text`,
    from the start of its paragraph to its closing brace."""
    out = []
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
    auxS = torch.empty(nS, 4, dtype=torch.float32, device=dev)
    gS = torch.empty_like(S.A)
    lamG = torch.empty(nG, 3, dtype=torch.float64, device=dev)
    auxG = torch.empty(nG, 4, dtype=torch.float64, device=dev)
    gG = torch.empty_like(G.A)
    wS, wG = S.extra["w"], G.extra["w"]
    stats = eig3.Stats(dev)

    def fwd_S():
        eig3.eigvals(S.A, precision="f32c", return_aux=True, out=lamS, aux_out=auxS, stats=stats)

    def bwd_S():
        eig3.eigvals_backward(S.A, wS, aux=auxS, precision="f32c", out=gS)

    def fwd_G():
        eig3.eigvals(G.A, precision="f64", return_aux=True, out=lamG, aux_out=auxG, stats=stats)

    def bwd_G():
        eig3.eigvals_backward(G.A, wG, aux=auxG, precision="f64", out=gG)

    # The two halves are independent.  The binary64 kernels keep the FP64 pipe
    # busy with little else; the compensated binary32 kernels use the FP32
    # pipes, so they run on a second stream beside them.  Launched eagerly (4
    # launches per step): replaying the same work as one CUDA graph measured
    # 70.8-72.6 ms per step from run to run, the eager launches a steady 70.6 ms
    # (the graph does not keep the binary64 kernels' blocks first on the SMs).
    s64, s32 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def step():
        s64.wait_stream(stream)
        s32.wait_stream(stream)
        with torch.cuda.stream(s64):
            fwd_G()
            bwd_G()
        with torch.cuda.stream(s32):
            fwd_S()
            bwd_S()
        stream.wait_stream(s64)
        stream.wait_stream(s32)

    launches_per_step = 4
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

    # ---- per-kernel durations (eager, same launches, events on the launch stream) ----
    kern = {}
    for name, fn in (("fwd_f32c_sym6", fwd_S), ("bwd_f32c_sym6", bwd_S),
                     ("fwd_f64_general9", fwd_G), ("bwd_f64_general9", bwd_G)):
        fn()
        kern[name] = timed(fn, args.steps, stream)
    pk, pk_src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_inst = sms * FP64_LANES_PER_SM * sm_max * 1e6 / 1e12      # T inst/s
    c = FWD_F64_COUNTERS
    fresh = kernel_source_md5(FWD_F64_SOURCES) == c["source_md5"]
    t_fwdG = kern["fwd_f64_general9"] * 1e-3
    achieved = c["fp64_pipe_inst"] * nG / t_fwdG / 1e12
    flop = 2 * c["dfma"] + c["dmul"] + c["dadd"]
    roofline = {"kernel": "k_eigvals<general9, f64, aux, stats> (binary64 forward, 2^27 matrices)",
                "bound": "alu", "unit": "T FP64-pipe inst/s", "achieved": achieved,
                "peak": peak_inst, "frac": achieved / peak_inst,
                "traffic": c["dram_bytes"] * nG if fresh else None,
                "counters_fresh": fresh,
                "peak_source": f"{sms} SMs x {FP64_LANES_PER_SM} FP64 lanes x {sm_max:.0f} MHz "
                               f"(unit counts and clock; MEASURED_PEAKS has no FP64 figure)",
                "algorithmic_per_matrix": {"fp64_pipe_inst": c["fp64_pipe_inst"], "dfma": c["dfma"],
                                           "dmul": c["dmul"], "dadd": c["dadd"],
                                           "hbm_bytes": 72 + 24 + 32},
                "flop_view": {"achieved_tflops": flop * nG / t_fwdG / 1e12,
                              "peak_tflops": 2 * peak_inst, "frac": flop * nG / t_fwdG / 1e12 /
                              (2 * peak_inst)},
                "hbm_view": {"achieved_gbs": (72 + 24 + 32) * nG / t_fwdG / 1e9,
                             "peak_gbs": pk.get("hbm_gbs"), "peak_source": pk_src,
                             "datasheet_gbs": 7900.0},
                "kernel_ms": kern}

    # ---- the other workloads' paths (fwd, fwd+bwd, FP64 vs compensated FP32) ----
    paths = {}
    if not args.skip_paths:
        paths = measure_paths(eig3, W, dev, stream, args.steps)

    # ---- end to end through host buffers (pinned), public API ----
    e2e = None
    if not args.skip_e2e:
        # page-locked host buffers per rank: inputs and outputs of both halves
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
                      "launch": "4 kernels per step, the binary32 pair on a second stream "
                                "beside the binary64 pair"},
           "roofline": roofline, "gpu_launches": launches_per_step * args.steps,
           "clocks": clocks.summary(), "e2e": e2e, "paths": paths,
           "stats": stats.read()}

    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only) ----
    if rank == 0 and world == 1 and not args.skip_cpu:
        out["cpu_baseline"], out["max_err_over_bound"] = cpu_baseline(
            eig3, S, G, lamS, lamG, gS, gG)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        tdist.destroy_process_group()
    return 0


def measure_paths(eig3, W, dev, stream, steps):
    paths = {}
    steps = max(steps, 3)
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


def measure_e2e(eig3, S, G, dev, stream, steps, shift=0):
    """The same step on host-resident data through the public API
    (paper_2511_00292_gb300.host.HostPipeline): the matrices and loss weights
    start in pinned host memory and the eigenvalues and gradients end there;
    every host-to-device and device-to-host copy is inside the timed region,
    overlapped with the kernels chunk by chunk on separate streams.  `shift`
    halves the batch that many times (host memory shared by several ranks)."""
    from paper_2511_00292_gb300.host import HostPipeline, pinned_copy, pinned_empty
    mS, mG = S.n >> shift, G.n >> shift
    hS = pinned_copy(S.A[:mS])
    hG = pinned_copy(G.A[:mG])
    hwS = pinned_copy(S.extra["w"][:mS])
    hwG = pinned_copy(G.extra["w"][:mG])
    olS = pinned_empty((mS, 3), torch.float32)
    olG = pinned_empty((mG, 3), torch.float64)
    ogS = pinned_empty(hS.shape, hS.dtype)
    ogG = pinned_empty(hG.shape, hG.dtype)
    h2d = sum(t.numel() * t.element_size() for t in (hS, hG, hwS, hwG))
    d2h = sum(t.numel() * t.element_size() for t in (olS, olG, ogS, ogG))
    pipe = HostPipeline(dev, chunk=1 << 21, depth=3)

    graph = pipe.capture([(hS, hwS, olS, ogS, None, "f32c"), (hG, hwG, olG, ogG, None, "f64")])

    def step():
        graph.replay()

    step()
    torch.cuda.synchronize(dev)
    k = max(1, min(steps, 3))
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
    del hS, hG, hwS, hwG, olS, olG, ogS, ogG, pipe
    return {"value": (mS + mG) / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "matrices_per_gpu": mS + mG,
            "mode": "pinned host buffers (host.pinned_empty: huge-page mappings registered "
                    "with CUDA), chunks of 2^21 streamed through 3 device slots "
                    "(H2D / kernels / D2H on 3 streams), captured once as a CUDA graph",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": k,
            "results_match_device": ok,
            "copy_roofline": {"both_directions_gbs_each": each_gbs, "floor_ms": floor_ms,
                              "frac": floor_ms / ms}}


def cpu_baseline(eig3, S, G, lamS, lamG, gS, gG):
    """The FP64 oracle (as it stands) on the host cores, on a bounded sample of
    the workload; the same sample gives the max error over the stability bound
    of the GPU results."""
    import oracle
    import workloads as W
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
    # accuracy of the GPU results on this sample
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
           "single_thread_ns_per_matrix": ns_1t}
    err = {"f32c_sym6": float(np.max(eS / bS)), "f64_general9": float(np.max(eG / bG)),
           "bound": "kappa ||A||_F u (u = 2^-24 for f32c, 2^-53 for f64; C = 1)",
           "sample_matrices": int(S64.shape[0] + G64.shape[0])}
    return cpu, err


KERNELS = ("fwd_f64_general9", "bwd_f64_general9", "fwd_f32c_sym6", "bwd_f32c_sym6",
           "fwd_f64_sym6", "mc_f64_sym6", "mc_f32c_sym6", "guard_f64_illcond",
           "proj_f32c_sym6")


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
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_single(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
