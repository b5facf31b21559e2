#!/usr/bin/env python
"""Benchmark of the KPM-DOS hot path (aug_spmmv) on GB300.

Workload: the 64x64x64 topological-insulator lattice of Eq. 1 (N =
1,048,576 rows, 13 non-zeros per row, disorder gamma = 1, seed 1), complex
double, M = 2000 moments from R = 32 random-phase vectors (1000 sweeps),
SELL-C-sigma with C = 32, sigma = 256.  One step = one full KPM-DOS run
(start vectors, the initial sweep, 999 aug_spmmv sweeps, eta reduction) on
inputs resident in HBM.  Every sweep moves 1.88 GB (> L2), so no flush is
needed between steps.

Reported (one JSON line on rank 0): algorithmic GB/s of the Eq. 4 traffic
model, the roofline of the sweep kernel timed alone with CUDA events, the
FP32-storage form on the same lattice shape (seed 2, M = 1024) with its
speed-up and moment / DOS error against the FP64 oracle, the end-to-end
rate through the host-buffer C calls, SM clocks sampled during the timed
region, and the CPU oracle timed on a bounded sample.

``--impl reference`` times the FP64 CPU oracle (the plain C reference of
the method) on the same workload and metric, one bounded sample per step.
"""
import argparse
import csv
import hashlib
import io
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from kpm_inputs import hamiltonians, workloads  # noqa: E402
from paper_1410_5242_gb300 import model  # noqa: E402

METRIC = "aug_spmmv HBM GB/s (frac of peak) and FP32/FP64 speedup at stated moment error"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 arithmetic peak derived from the unit counts: 2 FP64 FMA per clock per
# SM x 152 SMs x 2.07 GHz x 2 flops = 1.26 TFLOP/s (nominal 1.25).
FP64_PEAK_TFLOPS = 1.25
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "aug_spmmv_traffic.txt")
# the sources of each form's sweep kernel (the staged kernel in both forms
# at the bench's widths): the kernel files and, of kpm_internal.h, the
# device-side interface (error codes, producer records, StagedProblem,
# StagedParams); comments and blank lines do not count
KERNEL_SOURCES = {
    "fp64": ("aug_spmmv.cuh", "aug_spmmv_staged.cu", "kpm_internal.h"),
    "fp32": ("aug_spmmv.cuh", "aug_spmmv_staged.cu", "kpm_internal.h"),
}
INTERFACE_BEGIN = "#define KPM_DEVERR_TIMEOUT"
INTERFACE_END = "// The shared-memory layout of a staged launch"
# the launch helpers at the end of the staged kernel's file: occupancy queries
# and launches, which change no counter of the kernel
HOST_BEGIN = "// Host launch helpers: occupancy queries and launches, no device code."


def kernel_hash(form):
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[form]:
        text = open(os.path.join(ROOT, "paper_1410_5242_gb300", "csrc", f)).read()
        if f == "kpm_internal.h":
            text = text[text.index(INTERFACE_BEGIN):text.index(INTERFACE_END)]
        elif HOST_BEGIN in text:
            text = text[:text.index(HOST_BEGIN)]
        for line in text.splitlines():
            code = re.sub(r"//.*", "", line).rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:12]


def kernel_name(prec, launch, half=False):
    """The sweep kernel a launch shape runs (template arguments as built)."""
    real = "double" if prec == "fp64" else "float"
    if launch["stages"]:
        return "aug_spmmv_staged_kernel<%s,%d,%d,false,%s>, %d stages" % (
            real, launch["lanes_per_row"], launch["cols_per_lane"],
            "true" if half else "false", launch["stages"])
    return "aug_spmmv_kernel<%s,%d,%d>" % (real, launch["lanes_per_row"], launch["cols_per_lane"])


def measured_counter(form, name):
    """A per-launch counter of the form's sweep kernel from the committed ncu
    summary (profiles/aug_spmmv_traffic.txt), if it was taken on the current
    kernel sources (else None)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    vals = {}
    for line in open(TRAFFIC_FILE):
        parts = line.split()
        if len(parts) >= 2 and not line.startswith("#"):
            vals[parts[0]] = parts[1]
    if vals.get(form + "_kernel_hash") != kernel_hash(form):
        return None
    v = vals.get(form + "_" + name)
    return float(v) if v is not None else None


def measured_traffic(form):
    """DRAM bytes (read + write) per launch of the form's sweep kernel."""
    return measured_counter(form, "dram_bytes_per_launch")


def peaks():
    if os.path.exists(PEAKS_FILE):
        d = json.load(open(PEAKS_FILE))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def start(self):
        self.out = tempfile.TemporaryFile(mode="w+")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.out.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.out.read())) if len(r) >= 9]
        sm, smax, names = [], [], set()
        labels = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for lab, flag in zip(labels, r[5:9]):
                if flag.strip().lower() == "active":
                    names.add(lab)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(names), "samples": len(sm)}


# ------------------------------------------------------------ distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------- workloads
def ti_problem(cfg):
    h = hamiltonians.ti_hamiltonian(*cfg["dims"], gamma=cfg["gamma"], seed=cfg["seed"])
    from paper_1410_5242_gb300 import kpm
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    return h, a, b


def run_bytes(n, nnz, R, M, sd):
    """Eq. 4 for one KPM-DOS run: initial sweep (no W read) + M/2 - 1 sweeps."""
    return (model.sweep_bytes(n, nnz, R, sd, init=True)
            + (M // 2 - 1) * model.sweep_bytes(n, nnz, R, sd))


def time_steps(fn, steps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / steps


def kernel_only(ctx, R, launches, stream):
    """Average duration of the aug_spmmv sweep kernel alone: `launches`
    sweeps on resident blocks, no eta reduction, timed with CUDA events on
    the launching stream."""
    from kpm_inputs import vectors
    V = ctx.new_block(R)
    W = ctx.new_block(R)
    ctx.block_upload(R, vectors.random_phase_block(7, ctx.n, range(R)), V, stream=stream)
    bufs = [V, W]
    for i in range(3):
        ctx.aug_spmmv(R, bufs[i % 2], bufs[(i + 1) % 2], None, init=(i == 0), with_imag=False,
                      stream=stream)
    k = [3]

    def one():
        # the same kernel the moments path launches (no imaginary part)
        i = k[0]
        ctx.aug_spmmv(R, bufs[i % 2], bufs[(i + 1) % 2], None, with_imag=False, stream=stream)
        k[0] += 1

    return time_steps(one, launches, stream)


def oracle_sample(h, a, b, cols, M, seed):
    from oracle import oracle
    t0 = time.perf_counter()
    oracle.moments(h, a, b, M, seed, cols, threads=len(cols))
    return time.perf_counter() - t0


# ------------------------------------------------------------------ arms
def bench_ours(args, world, rank, local):
    import torch
    from paper_1410_5242_gb300 import build
    build.build()
    from paper_1410_5242_gb300 import kpm

    dev = local
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    hbm_peak, peak_src = peaks()
    cfg = workloads.TI_64
    M, R = cfg["M"], cfg["R"]
    seed = cfg["seed"] + rank  # replicas draw independent vectors
    h, a, b = ti_problem(cfg)
    n, nnz_h = h["n"], len(h["col"])

    ctx = kpm.create(h, a, b, precision=kpm.PREC_FP64, chunk_height=cfg["chunk_height"],
                     sigma=cfg["sigma"], device=dev)
    info = ctx.info()
    nnz = info["nnz"]
    eta_dev = torch.empty((R, M), dtype=torch.float64, device="cuda")

    def step():
        ctx.moments_device(M, R, seed, eta_dev, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(dev)
    clocks.start()
    launches0 = ctx.info()["kernel_launches"]
    t_step = time_steps(step, args.steps, stream)
    launches = ctx.info()["kernel_launches"] - launches0
    clock_info = clocks.stop()
    barrier(world)
    t_step = max_over_ranks(t_step, world)
    bytes_run = run_bytes(n, nnz, R, M, 16)
    value = world * bytes_run / t_step / 1e9

    # the sweep kernel alone (roofline of the dominant kernel)
    t_k = kernel_only(ctx, R, args.kernel_launches, stream)
    k_bytes = model.sweep_bytes(n, nnz, R, 16)
    # executed flops: the half-complex form skips the zero products
    half = bool(info["half_complex"])
    k_flops = model.fused_fp64_flops(nnz, n, R, half=half)
    achieved_tf = k_flops / t_k / 1e12
    k_gbs = k_bytes / t_k / 1e9
    traffic = measured_traffic("fp64")
    launch_shape = ctx.get_launch(R)

    # ---------------- FP32-storage form on the same lattice shape
    c4 = workloads.TI_64_FP32
    h4, a4, b4 = ti_problem(c4)
    M4, R4 = c4["M"], c4["R"]
    ctx32 = kpm.create(h4, a4, b4, precision=kpm.PREC_FP32, chunk_height=32, sigma=256, device=dev)
    eta32_dev = torch.empty((R4, M4), dtype=torch.float64, device="cuda")
    s32 = c4["seed"] + rank

    def step32():
        ctx32.moments_device(M4, R4, s32, eta32_dev, stream=stream)

    for _ in range(args.warmup):
        step32()
    t32 = time_steps(step32, args.steps, stream)
    t32 = max_over_ranks(t32, world)
    nnz4 = ctx32.info()["nnz"]
    bytes32 = run_bytes(h4["n"], nnz4, R4, M4, 8)
    t_k32 = kernel_only(ctx32, R4, args.kernel_launches, stream)
    k32_bytes = model.sweep_bytes(h4["n"], nnz4, R4, 8)
    k32_gbs = k32_bytes / t_k32 / 1e9
    traffic32 = measured_traffic("fp32")
    launch32 = ctx32.get_launch(R4)
    half32 = bool(ctx32.info()["half_complex"])

    fp32_err = None
    if rank == 0 and not args.skip_accuracy:
        fp32_err = fp32_accuracy(kpm, h4, a4, b4, c4, ctx32, dev, args)

    # ---------------- R sweep on the 64^3 lattice (code-balance drop, Eqs. 5-7)
    r_sweep = []
    if not args.skip_r_sweep:
        for Rs in workloads.R_SWEEP:
            t64 = kernel_only(ctx, Rs, max(3, args.kernel_launches // 10), stream)
            t32s = kernel_only(ctx32, Rs, max(10, args.kernel_launches // 2), stream)
            b64 = model.sweep_bytes(n, nnz, Rs, 16)
            b32 = model.sweep_bytes(h4["n"], nnz4, Rs, 8)
            # the widest column block's shape (complex double splits R = 64
            # into two 32-wide blocks): lanes per row x columns per lane,
            # blocks per SM, stages
            shape = {}
            for nm_, c_ in (("fp64", ctx), ("fp32", ctx32)):
                L = c_.get_launch(min(Rs, c_.max_block_width()))
                shape[nm_] = "%dx%d b%d s%d" % (L["lanes_per_row"], L["cols_per_lane"],
                                                L["blocks_per_sm"], L["stages"])
            entry = {
                "R": Rs, "B_min_fp64_bytes_per_flop": round(model.code_balance(nnz / n, Rs), 3),
                "fp64_ms": round(t64 * 1e3, 4), "fp64_GBs": round(b64 / t64 / 1e9, 1),
                "fp64_TFLOPs": round(model.fused_fp64_flops(nnz, n, Rs, half=half) / t64 / 1e12,
                                     4),
                "fp32_ms": round(t32s * 1e3, 4), "fp32_GBs": round(b32 / t32s / 1e9, 1),
                "fp32_frac_hbm": round(b32 / t32s / 1e9 / hbm_peak, 4), "shape": shape}
            if Rs >= 8:
                # the SELL layout kpm_autotune_layout picks for this width
                lay = kpm.autotune_layout(h4, a4, b4, Rs, precision=kpm.PREC_FP32, sweeps=3,
                                          device=dev)
                with kpm.create(h4, a4, b4, precision=kpm.PREC_FP32, device=dev,
                                chunk_height=lay["chunk_height"], sigma=lay["sigma"]) as ct:
                    tt = kernel_only(ct, Rs, max(10, args.kernel_launches // 2), stream)
                    bt = model.sweep_bytes(h4["n"], ct.info()["nnz"], Rs, 8)
                entry["fp32_tuned_layout"] = {
                    "chunk_height": lay["chunk_height"], "sigma": lay["sigma"],
                    "ms": round(tt * 1e3, 4), "frac_hbm": round(bt / tt / 1e9 / hbm_peak, 4)}
            r_sweep.append(entry)

    # ---------------- optimisation stages of the paper on this GPU
    ablation = None
    if not args.skip_ablation:
        ablation = ablation_stages(kpm, h, a, b, ctx, ctx32, n, nnz, h4["n"], nnz4, stream)

    # ---------------- the 64-problem ensemble in one graph launch
    ens = None
    if not args.skip_ensemble:
        ens = ensemble_rate(kpm, dev, args, stream, world, hbm_peak)

    # ---------------- A(k, E) through the device-built Bloch waves
    spectral = None
    if not args.skip_spectral:
        spectral = spectral_rate(kpm, ctx, h["dims"], n, nnz, stream)

    # ---------------- end to end through the host-buffer C calls
    e2e = None
    if not args.skip_e2e:
        e2e = e2e_rate(kpm, h, a, b, cfg, M, R, seed, dev, args.steps, world)

    # ---------------- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = cpu_baseline(h, a, b, cfg)

    # ---------------- the 240 x 240 x 120 lattice (N = 1 only: it holds ~60 GB)
    large = None
    if world == 1 and not args.skip_large:
        large = large_rate(kpm, stream, hbm_peak, peak_src)

    sweeps = M // 2
    out = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_step * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": "TI lattice 64x64x64 (N=%d, nnz=%d), complex double, M=%d, R=%d, "
                        "SELL-C-sigma C=%d sigma=%d, seed %d" % (n, nnz_h, M, R, cfg["chunk_height"],
                                                               cfg["sigma"], cfg["seed"]),
            "sweeps_per_step": sweeps,
            "bytes_per_step": bytes_run,
            "l2": "inputs larger than L2 (%.2f GB per sweep vs 129 MB)" % (k_bytes / 1e9),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "launch": launch_shape,
        },
        "frac_of_hbm_peak": round(value / world / hbm_peak, 4),
        "vector_updates_per_s": world * R * sweeps / t_step,
        "table1_gflops": world * sweeps * model.sweep_flops(n, nnz, R) / t_step / 1e9,
        "roofline": {
            "bound": "alu", "achieved": round(achieved_tf, 4), "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": round(achieved_tf / FP64_PEAK_TFLOPS, 4),
            "traffic": traffic,
            "traffic_source": traffic_source("fp64", traffic),
            # the FP64 pipe's busy fraction in the same ncu capture (the flop
            # count above leaves out the old-W subtraction and the 1/2 of the
            # initial sweep)
            "fp64_pipe_active_ncu": measured_counter("fp64", "fp64_pipe_active"),
            "kernel": kernel_name("fp64", launch_shape, half),
            "half_complex": half,
            "avg_launch_ms": round(t_k * 1e3, 4),
            "algorithmic_bytes": k_bytes, "algorithmic_flops": k_flops,
            "hbm_gbs": round(k_gbs, 1), "hbm_frac": round(k_gbs / hbm_peak, 4),
            "peak_source": "FP64 nominal (2 DFMA/clk/SM x 152 SMs x 2.07 GHz); HBM %s %.0f GB/s"
                           % (peak_src, hbm_peak),
        },
        "fp32_form": {
            "workload": "TI lattice 64x64x64, complex float storage, M=%d, R=%d, seed %d"
                        % (M4, R4, c4["seed"]),
            "value": round(world * bytes32 / t32 / 1e9, 2), "unit": "GB/s",
            "ms_per_step": round(t32 * 1e3, 3),
            "frac_of_hbm_peak": round(bytes32 / t32 / 1e9 / hbm_peak, 4),
            "speedup_per_sweep_vs_fp64": round((t_step / sweeps) / (t32 / (M4 // 2)), 3),
            "roofline": {"bound": "hbm", "achieved": round(k32_gbs, 1), "peak": hbm_peak,
                         "unit": "GB/s", "frac": round(k32_gbs / hbm_peak, 4),
                         "traffic": traffic32, "traffic_source": traffic_source("fp32", traffic32),
                         "avg_launch_ms": round(t_k32 * 1e3, 4),
                         "algorithmic_bytes": k32_bytes,
                         "kernel": kernel_name("fp32", launch32, half32),
                         "launch": launch32,
                         "peak_source": "HBM %s %.0f GB/s" % (peak_src, hbm_peak)},
            "accuracy": fp32_err,
        },
        "r_sweep": r_sweep,
        "ablation": ablation,
        "ensemble": ens,
        "spectral_function": spectral,
        "large": large,
        "e2e": e2e,
        "gpu_launches": launches * world,
        "clocks": clock_info,
        "cpu_baseline": cpu,
    }
    out["summary"] = summary(out)
    ctx.close()
    ctx32.close()
    if rank == 0:
        print(json.dumps(out))


def traffic_source(form, traffic):
    if traffic is None:
        return ("none: profiles/aug_spmmv_traffic.txt was taken on other kernel sources "
                "(hash %s now)" % kernel_hash(form))
    return "ncu record in profiles/aug_spmmv_traffic.txt, kernel hash %s" % kernel_hash(form)


def summary(out):
    """The figures the targets name, last on the line: the FP32-storage form's
    roofline fraction, speed-up and error, the FP64 form's pipe fraction, the
    240x240x120 lattice in both forms, the ensemble and the R sweep."""
    def r(x, k=4):
        return None if x is None else round(x, k)
    fp = out["fp32_form"]
    acc = fp.get("accuracy") or {}
    sm = {"fp64_sweep_frac_of_fp64_peak": out["roofline"]["frac"],
          "fp64_sweep_hbm_frac": out["roofline"]["hbm_frac"],
          "fp32_sweep_frac_of_hbm": fp["roofline"]["frac"],
          "fp32_sweep_ms": fp["roofline"]["avg_launch_ms"],
          "fp32_speedup_per_sweep_vs_fp64": fp["speedup_per_sweep_vs_fp64"],
          "fp32_max_abs_dmu_vs_oracle": acc.get("max_abs_dmu_vs_oracle"),
          "fp32_dos_l1_vs_oracle": acc.get("dos_l1_vs_oracle"),
          "fp32_max_abs_dmu_vs_gpu_fp64": acc.get("max_abs_dmu_vs_gpu_fp64"),
          "fp64_max_abs_dmu_vs_oracle": acc.get("fp64_form_max_abs_dmu_vs_oracle")}
    if out["r_sweep"]:
        sm["r_sweep_fp32_frac"] = {str(e["R"]): e["fp32_frac_hbm"] for e in out["r_sweep"]}
        sm["r_sweep_fp32_frac_tuned_layout"] = {
            str(e["R"]): e["fp32_tuned_layout"]["frac_hbm"] for e in out["r_sweep"]
            if "fp32_tuned_layout" in e}
    lg = out.get("large")
    if lg:
        sm["large_240x240x120"] = {
            "fp64_frac_of_fp64_peak": lg["fp64"].get("frac_of_fp64_peak"),
            "fp64_hbm_frac": lg["fp64"]["frac_of_hbm_peak"],
            "fp32_frac_of_hbm": lg["fp32"]["frac_of_hbm_peak"],
            "fp32_max_abs_dmu_vs_fp64": r(lg["fp32_max_abs_dmu_vs_fp64"], 12),
            "fp32_dos_l1_vs_fp64": r(lg["fp32_dos_l1_vs_fp64"], 9),
            "fp64_mu0_minus_1": r(lg["fp64"]["checks"]["mu0_minus_1"], 16)}
    if out.get("ensemble"):
        sm["ensemble_frac_of_hbm"] = out["ensemble"]["frac_of_hbm_peak"]
    return sm


def ablation_stages(kpm, h, a, b, ctx, ctx32, n, nnz, n4, nnz4, stream):
    """The paper's optimisation stages (Figs. 3-5, Table III, Fig. 10) on the
    64^3 lattice, R = 32, M = 400, timed with CUDA events: the naive
    library-call algorithm, fused aug_spmv in throughput mode (R runs of one
    vector), blocked aug_spmmv with a reduction after every sweep and with
    batched reductions, and the sweep kernel without dots / plain SpMMV."""
    import torch
    M, R, seed = 400, 32, 9
    eta = torch.empty((R, M), dtype=torch.float64, device="cuda")
    eta1 = torch.empty((1, M), dtype=torch.float64, device="cuda")
    out = {"M": M, "R": R, "unit": "ms per KPM-DOS run"}

    def timed(fn):
        fn()
        return time_steps(fn, 1, stream) * 1e3

    with kpm.Naive(h, a, b) as nv:
        out["fp64_naive_library_calls"] = round(timed(lambda: nv.moments_device(M, R, seed, eta,
                                                                                 stream=stream)), 2)
    for name, c in (("fp64", ctx), ("fp32", ctx32)):
        t1 = timed(lambda: c.moments_device(M, 1, seed, eta1, stream=stream))
        out[name + "_aug_spmv_throughput_mode"] = round(R * t1, 2)
        c.set_reduce_interval(1)
        out[name + "_aug_spmmv_reduce_every_sweep"] = round(
            timed(lambda: c.moments_device(M, R, seed, eta, stream=stream)), 2)
        c.set_reduce_interval(0)
        out[name + "_aug_spmmv"] = round(timed(lambda: c.moments_device(M, R, seed, eta,
                                                                         stream=stream)), 2)
        V, W = c.new_block(R), c.new_block(R)
        c.aug_spmmv(R, V, W, None, init=True, with_imag=False, stream=stream)
        for variant, label in ((2, "plain_spmmv"), (1, "aug_spmmv_no_dots"), (0, "aug_spmmv")):
            def sweeps():
                for _ in range(10):
                    c.sweep_variant(R, V, W, variant, stream=stream)
            out["%s_sweep_ms_%s" % (name, label)] = round(timed(sweeps) / 10, 4)
    naive = out["fp64_naive_library_calls"]
    out["fp64_speedup_vs_naive"] = {k: round(naive / out[k], 2) for k in (
        "fp64_aug_spmv_throughput_mode", "fp64_aug_spmmv_reduce_every_sweep", "fp64_aug_spmmv",
        "fp32_aug_spmmv")}
    sd_bytes = {"naive": model.kpm_traffic(M, n, nnz, R, 16, "naive"),
                "aug_spmv": model.kpm_traffic(M, n, nnz, R, 16, "aug_spmv"),
                "aug_spmmv": model.kpm_traffic(M, n, nnz, R, 16, "aug_spmmv")}
    out["fp64_eq4_bytes"] = sd_bytes
    return out


def ensemble_rate(kpm, dev, args, stream, world, hbm_peak):
    """The ensemble recipe (64 lattices 16..96 x 16..96 x 16..48, gamma in
    [0, 4], even M in [512, 4096], R in {8, 16, 32, 64}, complex float) as
    one kpm_batch: graph launches timed with CUDA events (setup excluded).
    Each block-width class takes the SELL chunk height and sorting window
    that kpm_autotune_layout picks on its largest problem."""
    probs = workloads.ensemble()
    t0 = time.perf_counter()
    hs = []
    for p in probs:
        h = hamiltonians.ti_hamiltonian(*p["dims"], gamma=p["gamma"], seed=p["seed"])
        a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
        hs.append((h, a, b))
    t_build = time.perf_counter() - t0
    # --ensemble-tuned: the layouts and launch shapes an earlier run chose
    # (its JSON line), for a run under a profiler, whose timings would steer
    # the autotuners elsewhere
    fixed = None
    if getattr(args, "ensemble_tuned", None):
        fixed = json.loads(open(args.ensemble_tuned).read().strip().splitlines()[-1])
    t0 = time.perf_counter()
    layout = {}
    for R in sorted(set(p["R"] for p in probs)):
        if fixed:
            L = fixed["tuned_layout"][str(R)]
            layout[R] = {"chunk_height": L["C"], "sigma": L["sigma"]}
            continue
        big = max((i for i, p in enumerate(probs) if p["R"] == R), key=lambda i: hs[i][0]["n"])
        h, a, b = hs[big]
        layout[R] = kpm.autotune_layout(h, a, b, R, precision=kpm.PREC_FP32, sweeps=3,
                                        device=dev)
    t_layout = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctxs, Ms, Rs, seeds = [], [], [], []
    for p, (h, a, b) in zip(probs, hs):
        L = layout[p["R"]]
        ctxs.append(kpm.create(h, a, b, precision=kpm.PREC_FP32, device=dev,
                               chunk_height=L["chunk_height"], sigma=L["sigma"]))
        Ms.append(p["M"])
        Rs.append(p["R"])
        seeds.append(p["seed"])
    t_setup = time.perf_counter() - t0 + t_build
    # autotune the launch shape of each block-width class on its largest
    # problem (kpm_autotune) and give it to the class's other problems: the
    # batch launches each class with its first problem's shape
    t0 = time.perf_counter()
    tuned = {}
    for R in sorted(set(Rs)):
        members = [c for c, r in zip(ctxs, Rs) if r == R]
        rep = max(members, key=lambda c: c.n)
        if fixed:
            shape = fixed["tuned_launch"][str(R)]
            rep = None
        else:
            rep.autotune(R, sweeps=3, stream=stream)
            shape = rep.get_launch(R)
        for c in members:
            if c is not rep:
                c.set_launch(R, shape["lanes_per_row"], shape["cols_per_lane"],
                             shape["block_threads"], shape["blocks_per_sm"],
                             shape["tile_groups"], shape["stages"])
        tuned[str(R)] = shape
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch = kpm.Batch(ctxs, Ms, Rs, seeds)
    t_capture = time.perf_counter() - t0
    info = batch.info()
    batch.launch(stream)  # warm-up run
    t = time_steps(lambda: batch.launch(stream), args.ensemble_runs, stream)
    t = max_over_ranks(t, world)
    gbs = info["algorithmic_bytes"] / t / 1e9
    eta0 = batch.eta(0)
    out = {"workload": "64 TI lattices (%d rows in total), complex float, one graph launch"
                       % sum(c.n for c in ctxs),
           "value": round(world * gbs, 1), "unit": "GB/s", "frac_of_hbm_peak": round(gbs / hbm_peak, 4),
           "ms_per_run": round(t * 1e3, 1), "runs": args.ensemble_runs, "warmup": 1,
           "algorithmic_bytes_per_run": info["algorithmic_bytes"], "sweeps": info["sweeps"],
           "steps": info["steps"], "graph_kernel_nodes": info["kernel_launches"],
           "classes": info["classes"], "staged_classes": info["staged_classes"],
           "setup_s": round(t_setup, 1), "autotune_s": round(t_tune, 1), "tuned_launch": tuned,
           "layout_autotune_s": round(t_layout, 1),
           "tuned_layout": {str(R): {"C": L["chunk_height"], "sigma": L["sigma"]}
                            for R, L in layout.items()},
           "capture_s": round(t_capture, 2),
           "mu0_problem0": float(kpm.eta_to_mu(eta0)[0])}
    batch.close()
    for c in ctxs:
        c.close()
    return out


def fp32_accuracy(kpm, h4, a4, b4, c4, ctx32, dev, args):
    """Per-moment and DOS error of the FP32-storage form: all 32 vectors
    against the GPU FP64 form, and the sampled vectors 0 and 1 directly
    against the FP64 CPU oracle."""
    from oracle import oracle
    M4, R4, s = c4["M"], c4["R"], c4["seed"]
    eta32 = ctx32.moments(M4, R4, s)
    with kpm.create(h4, a4, b4, precision=kpm.PREC_FP64, device=dev) as c64:
        eta64 = c64.moments(M4, R4, s)
    mu32, mu64 = kpm.eta_to_mu(eta32), kpm.eta_to_mu(eta64)
    K = 4096
    _, r32 = kpm.dos(mu32, K, a4, b4)
    _, r64 = kpm.dos(mu64, K, a4, b4)
    out = {"max_abs_dmu_vs_gpu_fp64": float(np.abs(mu32 - mu64).max()),
           "dos_l1_vs_gpu_fp64": float(np.abs(r32 - r64).sum() / np.abs(r64).sum()),
           "K": K}
    if not args.skip_oracle_accuracy:
        cols = [0, 1]
        ref, _ = oracle.moments(h4, a4, b4, M4, s, cols, threads=2)
        mu_o = oracle.eta_to_mu(ref)
        mu_g = kpm.eta_to_mu(eta32[cols])
        mu_g64 = kpm.eta_to_mu(eta64[cols])
        _, ro = oracle.dos(mu_o, K, a4, b4)
        _, rg = kpm.dos(mu_g, K, a4, b4)
        out.update({"sampled_vectors": cols,
                    "max_abs_dmu_vs_oracle": float(np.abs(mu_g - mu_o).max()),
                    "dos_l1_vs_oracle": float(np.abs(rg - ro).sum() / np.abs(ro).sum()),
                    "fp64_form_max_abs_dmu_vs_oracle": float(np.abs(mu_g64 - mu_o).max())})
    return out


def e2e_rate(kpm, h, a, b, cfg, M, R, seed, dev, steps, world):
    """Through the user's calls with host buffers: kpm_create (CSR -> SELL on
    the host, upload), kpm_moments (eta copied to host), kpm_destroy."""
    import torch
    steps = max(1, min(steps, 3))
    h2d = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        c = kpm.create(h, a, b, precision=kpm.PREC_FP64, chunk_height=cfg["chunk_height"],
                       sigma=cfg["sigma"], device=dev)
        info = c.info()
        c.moments(M, R, seed)
        c.close()
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / steps
    t = max_over_ranks(t, world)
    h2d = info["upload_bytes"]
    return {"value": round(world * run_bytes(h["n"], info["nnz"], R, M, 16) / t / 1e9, 2),
            "unit": "GB/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(M * R * 8),
            "steps": steps, "ms_per_step": round(t * 1e3, 1)}


def spectral_rate(kpm, ctx, dims, n, nnz, stream):
    """A(k, E) along a path of 8 Bloch vectors (Gamma -> X -> M -> R of the
    cubic lattice), 4 orbitals each (R = 32), M = 512, through
    kpm_moments_plane_wave with host output: start waves built on the
    device, CUDA events around each call."""
    import torch
    L = np.asarray(dims, dtype=np.float64)
    path = [(0, 0, 0), (0.25, 0, 0), (0.5, 0, 0), (0.5, 0.25, 0), (0.5, 0.5, 0),
            (0.5, 0.5, 0.25), (0.5, 0.5, 0.5), (0.25, 0.25, 0.25)]
    q = np.repeat(np.round(np.asarray(path) * L) / L, 4, axis=0)  # on the Bloch grid
    orb = np.tile(np.arange(4), len(path))
    M, R = 512, q.shape[0]
    ctx.moments_plane_wave(M, dims, 4, q, orb, stream=stream)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    runs = 3
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(runs):
        eta = ctx.moments_plane_wave(M, dims, 4, q, orb, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / runs
    mu0 = float(kpm.eta_to_mu(eta[:4])[0])
    return {"workload": "A(k,E) at 8 Bloch vectors x 4 orbitals (R = %d) of the 64^3 lattice, "
                        "M = %d, complex double" % (R, M),
            "value": round(run_bytes(n, nnz, R, M, 16) / t / 1e9, 1), "unit": "GB/s",
            "ms_per_run": round(t * 1e3, 2), "mu0_gamma": mu0}


def cpu_baseline(h, a, b, cfg):
    cores = os.cpu_count() or 1
    cols = list(range(min(cores, cfg["R"])))
    Ms = 40
    t = oracle_sample(h, a, b, cols, Ms, cfg["seed"])
    nnz = len(h["col"])
    return {"value": round(run_bytes(h["n"], nnz, len(cols), Ms, 16) / t / 1e9, 3),
            "unit": "GB/s", "cores": len(cols), "kind": "oracle",
            "sample": "%d vectors x %d moments (%d sweeps) of the 64^3 lattice, one vector per "
                      "thread, %.1f s" % (len(cols), Ms, Ms // 2, t),
            "vector_updates_per_s": len(cols) * (Ms // 2) / t}


def bench_reference(args, world, rank):
    """The FP64 CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    cfg = workloads.TI_64
    h = hamiltonians.ti_hamiltonian(*cfg["dims"], gamma=cfg["gamma"], seed=cfg["seed"])
    from oracle import oracle
    oracle.build()
    a, b = oracle.scale_from_bounds(*oracle.gershgorin(h), 0.01)
    cores = os.cpu_count() or 1
    cols = list(range(min(cores, cfg["R"])))
    Ms = 20
    for _ in range(args.warmup):
        oracle_sample(h, a, b, cols, 4, cfg["seed"])
    ts = [oracle_sample(h, a, b, cols, Ms, cfg["seed"]) for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    nnz = len(h["col"])
    value = run_bytes(h["n"], nnz, len(cols), Ms, 16) / t / 1e9
    sample = ("%d vectors x %d moments (%d sweeps) of the 64^3 lattice per step, one vector per "
              "thread" % (len(cols), Ms, Ms // 2))
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(t * 1e3, 1), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "TI lattice 64x64x64, complex double, M=%d, R=%d (sampled)"
                      % (cfg["M"], cfg["R"])},
           "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": len(cols),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def moment_checks(kpm, eta, eti):
    """Invariants of the moments that hold at any size (Sec. "Problem
    Description" and the recurrence of Eq. 3): mu_0 = 1, Im eta = 0 for a
    Hermitian H, eta_2m = <nu_m|nu_m> >= 0, and |c_n| <= eta_0 per vector
    (the spectrum of a(H - b) lies in [-1, 1])."""
    eta0 = eta[:, :1]
    c = eta.copy()
    c[:, 2::2] = 2 * eta[:, 2::2] - eta0
    c[:, 3::2] = 2 * eta[:, 3::2] - eta[:, 1:2]
    return {"mu0_minus_1": float(kpm.eta_to_mu(eta)[0] - 1.0),
            "max_abs_im_eta_over_eta0": float(np.abs(eti).max() / eta0.min()),
            "min_eta_even_over_eta0": float((eta[:, 0::2] / eta0).min()),
            "max_abs_c_over_eta0": float(np.abs(c / eta0).max())}


def large_rate(kpm, stream, hbm_peak, peak_src, launches64=5, launches32=20):
    """The 240 x 240 x 120 lattice (N = 27,648,000 rows, 359M entries, gamma
    = 2, seed 2; the single-GPU roofline workload): in both forms the sweep
    kernel alone at R = 32 (CUDA events on the launching stream) and one
    KPM-DOS run of M = 1024 moments through kpm_moments (host output), the
    invariants of the FP64 moments, and the FP32 form's moment and DOS
    error against them.  Parity against the CPU oracle on this lattice is a
    GPU test (columns 0, 1, 16, 31)."""
    import torch
    cfg = workloads.TI_LARGE
    t0 = time.perf_counter()
    h, a, b = ti_problem(cfg)
    t_build = time.perf_counter() - t0
    n, R, M, seed = h["n"], cfg["R"], cfg["M"], cfg["seed"]
    # rows in tiles of 240 x 24 sites through all z (kpm_options.row_order):
    # a V row's +z and -z uses are then one tile plane (0.9 MB of rows)
    # apart instead of a whole 240 x 240 plane, so the rows stay in L2
    # between them; the moments do not depend on the order
    nx, ny, nz = cfg["dims"]
    tile = (nx, cfg["tile_y"], nz)
    row_order = hamiltonians.cube_row_order(cfg["dims"], block=tile)
    out = {"workload": "TI lattice 240x240x120 (N=%d, nnz=%d), R=%d, M=%d, gamma=%g, seed %d; "
                       "rows in %dx%dx%d site tiles" % (n, len(h["col"]), R, M, cfg["gamma"], seed,
                                                        *tile),
           "lattice_build_s": round(t_build, 1)}
    etas = {}
    for name, prec, sd, launches in (("fp64", kpm.PREC_FP64, 16, launches64),
                                     ("fp32", kpm.PREC_FP32, 8, launches32)):
        t0 = time.perf_counter()
        ctx = kpm.create(h, a, b, precision=prec, row_order=row_order)
        t_create = time.perf_counter() - t0
        info = ctx.info()
        nnz = info["nnz"]
        t = kernel_only(ctx, R, launches, stream)
        byt = model.sweep_bytes(n, nnz, R, sd)
        entry = {"create_s": round(t_create, 1), "launch": ctx.get_launch(R),
                 "half_complex": bool(info["half_complex"]),
                 "avg_launch_ms": round(t * 1e3, 3), "algorithmic_bytes": byt,
                 "GBs": round(byt / t / 1e9, 1), "frac_of_hbm_peak": round(byt / t / 1e9 / hbm_peak, 4)}
        if prec == kpm.PREC_FP64:
            fl = model.fused_fp64_flops(nnz, n, R, half=bool(info["half_complex"]))
            entry["TFLOPs"] = round(fl / t / 1e12, 4)
            entry["frac_of_fp64_peak"] = round(fl / t / 1e12 / FP64_PEAK_TFLOPS, 4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eta, eti = ctx.moments(M, R, seed, imag=True, stream=stream)
        t_run = time.perf_counter() - t0
        entry["run_s"] = round(t_run, 3)
        entry["run_GBs"] = round(run_bytes(n, nnz, R, M, sd) / t_run / 1e9, 1)
        etas[name] = eta
        if prec == kpm.PREC_FP64:
            entry["checks"] = moment_checks(kpm, eta, eti)
        out[name] = entry
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
    mu64, mu32 = kpm.eta_to_mu(etas["fp64"]), kpm.eta_to_mu(etas["fp32"])
    _, r64 = kpm.dos(mu64, 4096, a, b)
    _, r32 = kpm.dos(mu32, 4096, a, b)
    out["fp32_max_abs_dmu_vs_fp64"] = float(np.abs(mu32 - mu64).max())
    out["fp32_dos_l1_vs_fp64"] = float(np.abs(r32 - r64).sum() / np.abs(r64).sum())
    out["peak_source"] = "HBM %s %.0f GB/s; FP64 %.2f TFLOP/s nominal" % (peak_src, hbm_peak,
                                                                         FP64_PEAK_TFLOPS)
    return out


def large_lattice(args):
    """--large: only the 240 x 240 x 120 lattice leg (see large_rate)."""
    import torch
    from paper_1410_5242_gb300 import build
    build.build()
    from paper_1410_5242_gb300 import kpm
    hbm_peak, peak_src = peaks()
    print(json.dumps({"large_lattice": large_rate(kpm, torch.cuda.current_stream(), hbm_peak,
                                                  peak_src)}))


def profile_sweeps(args):
    """A short program for ncu: 3 warm-up sweeps, then --kernel-launches
    sweeps of the 64^3 lattice at R = --profile-R (default 32) in one form,
    nothing else."""
    import torch
    from paper_1410_5242_gb300 import build
    build.build()
    from paper_1410_5242_gb300 import kpm
    cfg = workloads.TI_64 if args.profile_sweeps == "fp64" else workloads.TI_64_FP32
    h, a, b = ti_problem(cfg)
    prec = kpm.PREC_FP64 if args.profile_sweeps == "fp64" else kpm.PREC_FP32
    ctx = kpm.create(h, a, b, precision=prec, chunk_height=32, sigma=256)
    R = args.profile_R or cfg["R"]
    t = kernel_only(ctx, R, args.kernel_launches, torch.cuda.current_stream())
    print(json.dumps({"profile_sweeps": args.profile_sweeps, "R": R, "launch": ctx.get_launch(R),
                      "avg_launch_ms": round(t * 1e3, 4)}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel-launches", type=int, default=100)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--skip-oracle-accuracy", action="store_true")
    ap.add_argument("--skip-ensemble", action="store_true")
    ap.add_argument("--skip-r-sweep", action="store_true")
    ap.add_argument("--skip-ablation", action="store_true")
    ap.add_argument("--skip-spectral", action="store_true")
    ap.add_argument("--skip-large", action="store_true",
                    help="leave out the 240x240x120 lattice leg (a few minutes of host setup)")
    ap.add_argument("--ensemble-runs", type=int, default=1)
    ap.add_argument("--profile-R", type=int, default=0,
                    help="block width of --profile-sweeps (default: the workload's 32)")
    ap.add_argument("--profile-sweeps", choices=["fp32", "fp64"],
                    help="only run a few sweep launches of one form (for ncu captures)")
    ap.add_argument("--ensemble-only", action="store_true",
                    help="only the 64-problem ensemble (one warm-up and --ensemble-runs timed runs)")
    ap.add_argument("--ensemble-tuned", default=None,
                    help="with --ensemble-only: take the layouts and launch shapes from an "
                         "earlier --ensemble-only JSON line instead of autotuning")
    ap.add_argument("--large", action="store_true",
                    help="only the 240x240x120 lattice: the sweep kernel alone in both forms")
    args = ap.parse_args()
    if args.large:
        large_lattice(args)
        return
    if args.profile_sweeps:
        profile_sweeps(args)
        return
    if args.ensemble_only:
        import torch
        from paper_1410_5242_gb300 import build
        build.build()
        from paper_1410_5242_gb300 import kpm
        print(json.dumps(ensemble_rate(kpm, 0, args, torch.cuda.current_stream(), 1, peaks()[0])))
        return
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        bench_reference(args, world, rank)
    else:
        bench_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
