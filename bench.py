#!/usr/bin/env python3
"""Benchmark of the FFT-based quasi-periodic Green's function path on GB300.

Workload (the 3D doubly quasi-periodic G_d configuration): k = 2.5,
alpha = (0.1, 0.3), grid 128 x 128 x 64, 10^6 targets with x1, x2 ~ U[0, 2 pi),
x3 ~ U[-1, 1] (lattice points excluded within 1e-3), seed = rank.

One step = the whole path: gf_plan (double-precision coefficients fused into the
first inverse-FFT pass, the remaining FFT passes, the far-series table) plus
gf_eval_points over all targets (near gather + singular part + phase, far
eigen-series).  `value` = targets / device time per step (evals/s), double
precision (complex128) throughout; the split-precision path is reported beside
it.  L2 is flushed (256 MiB write) between timed steps.

--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1801_05977_gb300 import workloads as W  # noqa: E402

K_WAVE, ALPHA, GRID, N_TARGETS = 2.5, (0.1, 0.3), (128, 128, 64), 1_000_000
METRIC = "G_d evals/s on 1 GB300 at stated rel err; batched & surrogate vs plain FFT path"
WORKLOAD = "3D doubly quasi-periodic G_d, k=2.5, alpha=(0.1,0.3), grid 128x128x64, 1e6 uniform targets"
# The far series of a double-precision plan (three precision tiers by term
# size): the core (b|x3| <= Y0 = 18) is summed in double for the terms within
# e^-8 of the largest (b <= bmin + 8/|x3|, the double band) and in float-float
# on the FP32 pipe beyond (the float-float band); the rest (up to the
# truncation) is the float tail, summed by a concurrent kernel.  Work per term
# as the kernels implement it (an FMA counts 2 flops):
#   double band: y = b|x3| + ln b (1 FMA), r = y - y_j (1 add), e^{-r} to degree
#     3 (3 FMAs; table step 1/4096), one Reinsch step (2 FMAs + 1 add): 14 FP64 flops;
#   float-float band: the same steps in float pairs (TwoSum / FMA products):
#     86 FP32 instructions of which 12 FMAs = 98 FP32 flops;
#   float tail: one Horner step, b^2 = c1^2 + c2^2 - k^2 (1 FMA), b = b^2 rsqrt(b^2)
#     (1 mul), -b|x3| log2 e (1 mul), w = e/b (1 mul), complex step (2 FMA +
#     1 FMA + 1 mul), the test and the index (2): 14 FP32 flops (and 2 MUFU ops,
#     not counted).
FP64_TERM_FLOPS = 14
FF_TERM_FLOPS = 98
TAIL_TERM_FLOPS = 14
FAR_CORE_Y0 = 18.0
FAR_FF_GAP = 8.0
# DRAM bytes of one far3d_f64 launch on this workload: ncu (dram__bytes_read.sum
# + dram__bytes_write.sum) of a 2e5-target launch, scaled by the far targets
FAR_TRAFFIC_BYTES = 9.309696e6 * 5
# unit-count peaks, reported beside the measured ones (152 SMs, 2.07 GHz):
# FP64 2 FMA/clk/SM, FP32 128 FMA/clk/SM
# in-plane points of the far-region grid of the split leg that uses it
FAR_GRID_M = 512
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def disk_count(R2: np.ndarray, alpha) -> int:
    """Number of n in Z^2 with |alpha + n|^2 <= R2, summed over the entries of R2."""
    if R2.size == 0:
        return 0
    R = np.sqrt(R2.max())
    total = 0
    for n1 in range(int(np.floor(-alpha[0] - R)) - 1, int(np.ceil(-alpha[0] + R)) + 2):
        rem = R2 - (alpha[0] + n1) ** 2
        ok = rem >= 0
        s = np.sqrt(np.where(ok, rem, 0.0))
        lo = np.ceil(-alpha[1] - s)
        hi = np.floor(-alpha[1] + s)
        total += int(np.where(ok, np.maximum(hi - lo + 1, 0), 0).sum())
    return total


def smallest_evanescent_beta(k: float, alpha) -> float:
    """min |beta_n| over the n with |alpha_n| > k (attained next to the circle |alpha_n| = k)."""
    R = int(np.ceil(k)) + 3
    n = np.arange(-R - 1, R + 2)
    c1 = alpha[0] + n[:, None]
    c2 = alpha[1] + n[None, :]
    a2 = c1 * c1 + c2 * c2
    return float(np.sqrt(a2[a2 > k * k] - k * k).min())


def far_terms(x: np.ndarray, k: float, alpha, c: float, tol: float):
    """(all terms, core terms, {"double": double-band terms, "float-float": float-float-band
    terms}) of the far branch, each target with its own truncation, core and band radii."""
    z = np.abs(x[:, 2])
    z = z[z > c]
    T = np.log(1.0 / tol) + 3.0
    R2 = k * k + (T / z) ** 2
    Rc2 = np.minimum(k * k + (FAR_CORE_Y0 / z) ** 2, R2)
    bmin = smallest_evanescent_beta(k, alpha)
    Rd2 = np.minimum(k * k + (bmin + FAR_FF_GAP / z) ** 2, Rc2)
    n_core, n_double = disk_count(Rc2, alpha), disk_count(Rd2, alpha)
    return disk_count(R2, alpha), n_core, {"double": n_double, "float-float": n_core - n_double}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while the timed
    regions run (the double-precision, split and host-buffer steps)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler is producing lines
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:
                time.sleep(0.01)
            self.skip = len(self.lines)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "skip", 0):]:
            p = [s.strip() for s in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(vals, dev=None):
    """Entry-wise max over all ranks of a list of floats (identity on one rank).
    The timing rule of the multi-GPU line: every rank times the same steps and
    the job's time is the slowest rank's."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling)."""
    return world * units_per_rank / seconds


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# --------------------------------------------------------------------------- CPU oracle leg
def _oracle_problem():
    from oracle import oracle as O
    return O, O.Problem(dim=3, k=K_WAVE, alpha=ALPHA, M=GRID)


def oracle_full(x: np.ndarray):
    """The FP64 oracle as it stands, on all of this host's cores: the full plan
    (coefficients + naive O(M^2) DFT) and every target of the workload, the near
    and far branches timed apart; then one thread on a bounded sample (2000 near,
    200 far targets).  Returns (oracle output (n, 1), timing dict)."""
    O, pb = _oracle_problem()
    cores = O.set_threads(host_cores())
    t0 = time.perf_counter()
    g = O.grid(pb)
    t_plan = time.perf_counter() - t0
    far = np.abs(x[:, 2]) > pb.c
    ref = np.empty((x.shape[0], 1), dtype=np.complex128)
    t0 = time.perf_counter()
    ref[~far] = O.evaluate(pb, g, x[~far], O.OUT_GD)
    t_near = time.perf_counter() - t0
    t0 = time.perf_counter()
    ref[far] = O.evaluate(pb, g, x[far], O.OUT_GD)
    t_far = time.perf_counter() - t0
    n_near, n_far = int((~far).sum()), int(far.sum())
    O.set_threads(1)
    xs_near, xs_far = x[~far][:2000], x[far][:200]
    t0 = time.perf_counter()
    O.evaluate(pb, g, xs_near, O.OUT_GD)
    t1_near = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.evaluate(pb, g, xs_far, O.OUT_GD)
    t1_far = time.perf_counter() - t0
    O.set_threads(cores)
    info = {"cores": cores, "t_plan_s": t_plan, "t_near_s": t_near, "t_far_s": t_far, "n_near": n_near,
            "n_far": n_far, "near_evals_per_s": n_near / t_near, "far_evals_per_s": n_far / t_far,
            "eval_evals_per_s": x.shape[0] / (t_near + t_far),
            "one_thread": {"near_evals_per_s": xs_near.shape[0] / t1_near,
                           "far_evals_per_s": xs_far.shape[0] / t1_far,
                           "sample": f"{xs_near.shape[0]} near + {xs_far.shape[0]} far targets"}}
    return ref, info


def oracle_sample(n_sample: int, seed: int = 0):
    """One step of the reference arm: the full plan (coefficients + naive DFT)
    and a sample of n_sample of the workload's targets on all host cores.
    Returns (the whole workload's evals/s estimated from the step: plan + the
    sample's evaluation time scaled to 1e6 targets, measured step seconds, info)."""
    O, pb = _oracle_problem()
    cores = O.set_threads(host_cores())
    x = W.targets_3d(N_TARGETS, seed=seed)
    rng = np.random.default_rng(seed)
    xs = x[rng.choice(N_TARGETS, n_sample, replace=False)]
    t0 = time.perf_counter()
    g = O.grid(pb)
    t_plan = time.perf_counter() - t0
    t1 = time.perf_counter()
    O.evaluate(pb, g, xs, O.OUT_GD)
    t_eval = time.perf_counter() - t1
    step_s = time.perf_counter() - t0
    est = N_TARGETS / (t_plan + t_eval * (N_TARGETS / n_sample))
    return est, step_s, {"t_plan_s": t_plan, "t_eval_sample_s": t_eval, "sample_targets": n_sample, "cores": cores}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    vals, steps_s = [], []
    info = {}
    for i in range(args.warmup + args.steps):
        v, st, info = oracle_sample(args.ref_sample, seed=0)
        if i >= args.warmup:
            vals.append(v)
            steps_s.append(st)
    value = float(np.mean(vals))
    sample = (f"per step: the full plan (coefficients + naive O(M^2) DFT) and {args.ref_sample} of the 1e6 "
              f"targets, all host cores; value = 1e6 / (plan time + the sample's eval time x 1e6/"
              f"{args.ref_sample}); ms_per_step is the measured time of that step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(steps_s)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": N_TARGETS, "targets_per_step": args.ref_sample,
                   "precision": "fp64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": info["cores"], "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def measured_peak(key: str, fallback: float) -> tuple[float, str]:
    """A peak from MEASURED_PEAKS.json beside this file (the machine's measured HBM copy
    rate and cuBLAS bf16 rates), else the stated fallback; returns (value, which)."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def measure_peaks(dev):
    """FP64 and FP32 FMA rates of this GPU (gf_peak_probe, CUDA events, best of 3
    launches of about 40 ms each after one warm-up)."""
    import torch

    from paper_1801_05977_gb300 import gf

    sink = torch.zeros(2, dtype=torch.float64, device=dev)
    out = {}
    for name, pipe, iters in (("fp64", gf.GF_PROBE_FP64, 1500), ("fp32", gf.GF_PROBE_FP32, 80000)):
        best = 0.0
        for i in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fl = gf.peak_probe(pipe, iters, sink)
            e1.record()
            torch.cuda.synchronize()
            if i > 0:
                best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        out[name] = best
    # pipe overlap: FP64 chains on half the warps, FP32 chains on the other half,
    # each half alone and both at once (best of 3 after one warm-up, ms)
    ov = {}
    for name, pipe in (("fp64_half_ms", gf.GF_PROBE_FP64_HALF), ("fp32_half_ms", gf.GF_PROBE_FP32_HALF),
                       ("both_ms", gf.GF_PROBE_BOTH_HALVES)):
        best = None
        for i in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gf.peak_probe(pipe, 600, sink)
            e1.record()
            torch.cuda.synchronize()
            if i > 0:
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
        ov[name] = best
    ov["overlap"] = (ov["fp64_half_ms"] + ov["fp32_half_ms"] - ov["both_ms"]) / min(ov["fp64_half_ms"], ov["fp32_half_ms"])
    ov["note"] = ("gf_peak_probe halves: overlap = (t64 + t32 - t_both) / min(t64, t32): 1 when the pipes run "
                  "side by side, 0 when their times add")
    out["overlap"] = ov
    return out


# --------------------------------------------------------------------------- GPU leg
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1801_05977_gb300 import gf

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gf.lib()
    gf.set_phase_timing(True)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n_targets = args.targets
    x_np = W.targets_3d(n_targets, seed=rank)
    x = torch.from_numpy(x_np).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def run_path(precision: int, steps: int, warmup: int, tol: float, **extra):
        cdt = torch.complex128 if precision == gf.GF_FP64 else torch.complex64
        out = torch.empty((n_targets, 1), dtype=cdt, device=dev)
        kw = dict(precision=precision, series_tol=tol, **extra)
        for _ in range(warmup):
            p = gf.Plan(3, K_WAVE, ALPHA, GRID, **kw)
            p.eval_points_into(x, out, gf.GF_OUT_GD)
            torch.cuda.synchronize()
            p.close()
        times, phases = [], []
        l0 = gf.launch_count()
        for _ in range(steps):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p = gf.Plan(3, K_WAVE, ALPHA, GRID, **kw)
            p.eval_points_into(x, out, gf.GF_OUT_GD)
            e1.record(stream)
            barrier()
            times.append(e0.elapsed_time(e1))
            phases.append(p.phase_ms())
            p.close()
        launches = (gf.launch_count() - l0) / steps
        return out, times, phases, launches

    tol64 = 1e-16

    def path_line(name, t, ph):
        # profiling modes: one line with the device time per step and its phases
        print(json.dumps({"path": name, "targets": n_targets, "ms_per_step": float(np.mean(t)),
                          "phases_ms": {"synthesis": float(np.mean([p[0] for p in ph])),
                                        "near": float(np.mean([p[2] for p in ph])),
                                        "far": float(np.mean([p[3] for p in ph]))}}))

    if args.paths == "split":
        _, t, ph, _ = run_path(gf.GF_FP32_SPLIT, args.steps, args.warmup, 1e-8)
        path_line("split", t, ph)
        return 0
    if args.paths == "split_far_grid":
        _, t, ph, _ = run_path(gf.GF_FP32_SPLIT, args.steps, args.warmup, 1e-8, far_grid_M=FAR_GRID_M)
        path_line("split_far_grid", t, ph)
        return 0
    clk = ClockSampler(local).__enter__()
    out64, t64, ph64, launches = run_path(gf.GF_FP64, args.steps, args.warmup, tol64)
    if args.paths == "fp64":
        clk.__exit__()
        path_line("fp64", t64, ph64)
        return 0
    out32, t32, ph32, _ = run_path(gf.GF_FP32_SPLIT, args.steps, args.warmup, 1e-8)
    # split precision with the far-region grid (512 x 512 planes over c < |x3| <= c~)
    outfg, tfg, phfg, _ = run_path(gf.GF_FP32_SPLIT, args.steps, args.warmup, 1e-8, far_grid_M=FAR_GRID_M)

    ms64, ms32, msfg = max_over_ranks([np.mean(t64), np.mean(t32), np.mean(tfg)], dev)
    value = whole_job_rate(n_targets, world, ms64 * 1e-3)

    # e2e through the host-buffer entry point (pinned buffers, copies inside the timed region)
    x_pin = torch.from_numpy(x_np).pin_memory()
    o_pin = torch.empty((n_targets, 1), dtype=torch.complex128).pin_memory()
    e2e_t = []
    for i in range(0 if args.no_e2e else args.warmup + args.steps):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        p = gf.Plan(3, K_WAVE, ALPHA, GRID, precision=gf.GF_FP64, series_tol=tol64)
        p.eval_points_host(x_pin, o_pin, gf.GF_OUT_GD)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        p.close()
        if i >= args.warmup:
            e2e_t.append(dt)
    clk.__exit__()
    clocks = clk.summary()
    e2e_s = max_over_ranks([np.mean(e2e_t) if e2e_t else float("nan")], dev)[0]

    # roofline of the dominant kernels (the far series of the double-precision plan:
    # far3d_f64 and its concurrent float-tail kernel far3d_tail), two pipes
    far_ms = float(np.mean([p[3] for p in ph64]))
    near_ms = float(np.mean([p[2] for p in ph64]))
    synth_ms = float(np.mean([p[0] for p in ph64]))
    table_ms = float(np.mean([p[1] for p in ph64]))
    n_far_t = int((np.abs(x_np[:, 2]) > 0.6).sum())
    n_near_t = n_targets - n_far_t
    terms, core_terms, bands = far_terms(x_np, K_WAVE, ALPHA, 0.6, tol64)
    tail_terms = terms - core_terms
    peaks = measure_peaks(dev)
    w64 = world * FP64_TERM_FLOPS * bands["double"]
    w32 = world * (FF_TERM_FLOPS * bands["float-float"] + TAIL_TERM_FLOPS * tail_terms)
    t_far = far_ms * 1e-3
    # FP64-equivalent work: FP32 flops weighted by the measured rate ratio, so that
    # frac = W64 / (P64 t) + W32 / (P32 t), the share of the far phase the two pipes
    # would need for the term work at their measured rates
    w_eq = w64 + w32 * (peaks["fp64"] / peaks["fp32"])
    achieved = w_eq / t_far / 1e12
    frac64, frac32 = w64 / t_far / 1e12 / peaks["fp64"], w32 / t_far / 1e12 / peaks["fp32"]

    # split-precision error vs the double-precision path on this workload
    d = (out32.to(torch.complex128) - out64).abs()
    split_err = float(d.max() / out64.abs().max())
    far_mask = x[:, 2].abs() > 0.6
    dfg = (outfg.to(torch.complex128) - out64).abs()
    fg_err, fg_err_far = float(dfg.max() / out64.abs().max()), float(dfg[far_mask].max() / out64.abs().max())
    del dfg, d
    g64, g32 = out64.cpu().numpy(), out32.to(torch.complex128).cpu().numpy()

    batched = None if args.no_batch else run_batched(args, dev, flush)
    surrogate = None if args.no_surrogate else run_surrogate(args, dev)
    configs = None if args.no_configs else run_configs(args, dev, flush)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu, err_oracle = None, None
    if world == 1 and not args.no_cpu_baseline:
        ref, info = oracle_full(x_np)
        t_step = info["t_plan_s"] + info["t_near_s"] + info["t_far_s"]
        cpu = {"value": n_targets / t_step, "unit": "evals/s", "cores": info["cores"], "kind": "oracle",
               "sample": f"the whole workload, once: full plan (coefficients + naive O(M^2) DFT, "
                         f"{info['t_plan_s']:.1f} s) + all {n_targets} targets ({info['n_near']} near in "
                         f"{info['t_near_s']:.2f} s, {info['n_far']} far in {info['t_far_s']:.1f} s)",
               "eval_only": info["eval_evals_per_s"], "near_evals_per_s": info["near_evals_per_s"],
               "far_evals_per_s": info["far_evals_per_s"], "one_thread": info["one_thread"],
               "plan_s_naive_dft": info["t_plan_s"]}
        sc = np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())
        err_oracle = {"targets": n_targets,
                      "fp64": {"pointwise_max": float((np.abs(g64 - ref) / sc).max()),
                               "normwise": float(np.abs(g64 - ref).max() / np.abs(ref).max())},
                      "split": {"pointwise_max": float((np.abs(g32 - ref) / sc).max()),
                                "normwise": float(np.abs(g32 - ref).max() / np.abs(ref).max())},
                      "note": "every target of the step against the FP64 oracle; pointwise floor 1e-6 max|G|"}
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": world * n_targets, "precision": "fp64 (complex128)",
                   "series_tol": tol64, "parallelism": f"replicas{world}", "l2": "flushed (256 MiB write) between steps"},
        "phases_ms": {"synthesis": synth_ms, "near": near_ms, "far": far_ms,
                      "far_series_terms": terms, "far_core_terms": core_terms},
        "rates": {"plan_ms": synth_ms + table_ms,
                  "eval_only_evals_per_s": n_targets / ((near_ms + far_ms) * 1e-3),
                  "near_evals_per_s": n_near_t / (near_ms * 1e-3), "far_evals_per_s": n_far_t / (far_ms * 1e-3),
                  "note": "from the step's phase events (CUDA events on the plan's stream): plan = coefficients, "
                          "inverse FFTs and the far-series tables; eval = near pass (classification and gather) + "
                          "far pass; near and far rates over the targets of each branch"},
        "split": {"value": whole_job_rate(n_targets, world, ms32 * 1e-3), "ms_per_step": ms32, "dtype": "f32/f64 split",
                  "series_tol": 1e-8, "max_err_vs_fp64_normwise": split_err,
                  "phases_ms": {"synthesis": float(np.mean([p[0] for p in ph32])),
                                "near": float(np.mean([p[2] for p in ph32])),
                                "far": float(np.mean([p[3] for p in ph32]))}},
        "split_far_grid": {"value": whole_job_rate(n_targets, world, msfg * 1e-3), "ms_per_step": msfg,
                           "dtype": "f32/f64 split", "far_grid": f"{FAR_GRID_M}x{FAR_GRID_M} in-plane x 16 "
                                                                 f"intervals over 0.6 < |x3| <= 1",
                           "max_err_vs_fp64_normwise": fg_err, "far_targets_err_vs_fp64_normwise": fg_err_far,
                           "phases_ms": {"synthesis": float(np.mean([p[0] for p in phfg])),
                                         "near_and_far_grid": float(np.mean([p[2] for p in phfg])),
                                         "far_series": float(np.mean([p[3] for p in phfg]))}},
        "roofline": {"bound": "alu", "kernel": "far3d_f64 + far3d_tail (concurrent)", "achieved": achieved,
                     "peak": peaks["fp64"], "unit": "TFLOP/s (FP64-equivalent)", "frac": achieved / peaks["fp64"],
                     "traffic": FAR_TRAFFIC_BYTES if n_targets == 1_000_000 and FAR_TRAFFIC_BYTES else None,
                     "peaks_measured": {"fp64_tflops": peaks["fp64"], "fp32_tflops": peaks["fp32"],
                                        "how": "gf_peak_probe FMA chains, CUDA events, best of 3"},
                     "pipe_overlap": peaks["overlap"],
                     "peaks_nominal": {"fp64_tflops": FP64_NOMINAL_TFLOPS, "fp32_tflops": FP32_NOMINAL_TFLOPS},
                     "work": {"fp64_flops": w64, "fp32_flops": w32, "double_band_terms": bands["double"],
                              "float_float_terms": bands["float-float"], "tail_terms": tail_terms,
                              "all_terms": terms},
                     "frac_fp64_pipe": frac64, "frac_fp32_pipe": frac32,
                     "frac_max_model": max(frac64, frac32),
                     "note": "two-pipe roofline of the far phase over all series terms: achieved = (FP64 term "
                             "flops + FP32 term flops x P64/P32) / far-phase time, peak = measured FP64 rate, so "
                             "frac = W64/(P64 t) + W32/(P32 t); per term 14 FP64 flops (double band), 98 FP32 "
                             "flops (float-float band), 14 FP32 flops (float tail); frac_max_model takes the "
                             "busier pipe alone"},
        "err_vs_oracle": err_oracle,
        "e2e": {"value": whole_job_rate(n_targets, world, e2e_s), "unit": "evals/s",
                "h2d_bytes_per_step": int(x_np.nbytes), "d2h_bytes_per_step": int(n_targets * 16)},
        "batched": batched,
        "surrogate": surrogate,
        "other_configs": configs,
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batched(args, dev, flush):
    """Batched sweep: 256 (alpha, k) pairs, k ~ U[0.5, 5], alpha ~ U[-1/2, 1/2]^2
    (Wood gap 1e-3), grid per pair clamp(nextpow2(ceil(32 k)), 32, 256)^2 x 64,
    1e5 targets per pair, split precision.  Timed: the whole sweep (synthesis of
    every pair + evaluation of every target) as one CUDA graph, against the
    plain path called pair after pair (gf_plan + gf_eval_points)."""
    import torch

    from paper_1801_05977_gb300 import gf

    npairs, per = args.batch_pairs, args.batch_targets
    pr = W.sweep_pairs(npairs, seed=0)
    k = pr[:, 2].copy()
    al = pr[:, :2].copy()
    m = np.clip(2 ** np.ceil(np.log2(np.ceil(32 * k))), 32, 256).astype(np.int32)
    M = np.stack([m, m, np.full(npairs, 64, np.int32)], axis=1)
    xs = [W.targets_3d(per, seed=1000 + i) for i in range(npairs)]
    off = np.arange(npairs + 1, dtype=np.int64) * per
    x = torch.from_numpy(np.concatenate(xs)).to(dev)
    out = torch.empty((npairs * per, 1), dtype=torch.complex64, device=dev)
    t0 = time.perf_counter()
    batch = gf.Batch(k, al, M, precision=gf.GF_FP32_SPLIT)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    tune = batch.autotune(x, off, out, gf.GF_OUT_GD)
    s = torch.cuda.Stream(device=dev)
    times = []
    l0 = gf.launch_count()
    with torch.cuda.stream(s):
        for i in range(args.warmup + args.steps):
            flush.zero_()
            s.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            batch.run_graph(x, off, out, gf.GF_OUT_GD, stream=s)
            e1.record(s)
            s.synchronize()
            if i >= args.warmup:
                times.append(e0.elapsed_time(e1))
    graph_launches = (gf.launch_count() - l0) / (args.warmup + args.steps)
    ms_b = float(np.mean(times))
    # the synthesis alone (the three batched passes), against its algorithmic bytes:
    # per pair the first pass writes the work planes W, the x2 pass reads and writes
    # them, the x1 pass reads them and writes the padded gather grid G (W = G times
    # M1 M2 / ((M1 + 3)(M2 + 3)), the planes being those G keeps)
    syn = []
    with torch.cuda.stream(s):
        for i in range(args.warmup + args.steps):
            flush.zero_()
            s.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            batch.synthesize(stream=s)
            e1.record(s)
            s.synchronize()
            if i >= args.warmup:
                syn.append(e0.elapsed_time(e1))
    ms_syn = float(np.mean(syn))
    syn_bytes = 0.0
    for i in range(npairs):
        info = gf.PlanInfo()
        gf.lib().gf_plan_get_info(batch.plan_handle(i), ctypes.byref(info))
        G = float(info.grid_device_bytes)
        syn_bytes += 4.0 * G * info.M[0] * info.M[1] / ((info.M[0] + 3) * (info.M[1] + 3)) + G
    hbm, hbm_how = measured_peak("hbm_gbs", 6800.0)
    # plain path, pair after pair (one pass)
    ref = torch.empty_like(out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(npairs):
        p = gf.Plan(3, float(k[i]), tuple(al[i]), tuple(int(v) for v in M[i]), precision=gf.GF_FP32_SPLIT)
        p.eval_points_into(x[off[i]:off[i + 1]], ref[off[i]:off[i + 1]], gf.GF_OUT_GD)
        torch.cuda.synchronize()
        p.close()
    t_seq = time.perf_counter() - t0
    d = (out - ref).abs().max().item() / ref.abs().max().item()
    batch.close()
    total = npairs * per
    return {"value": total / (ms_b * 1e-3), "unit": "evals/s", "ms_per_step": ms_b, "pairs": npairs,
            "targets_per_pair": per, "grid_points_per_pair": "clamp(nextpow2(ceil(32k)),32,256)^2 x 64",
            "precision": "f32/f64 split", "launch": "one CUDA graph: 3 synthesis + memset + 4 eval kernels (classification, near list, far sort, far)",
            "graph_kernels_per_step": graph_launches, "tuning": {"tj_max": tune[0], "far_block": tune[1],
                                                                  "far_ctas_per_sm": tune[2]},
            "sequential_plain": {"value": total / t_seq, "s_per_sweep": t_seq,
                                 "how": "gf_plan + gf_eval_points pair after pair, wall clock"},
            "speedup_vs_sequential": (total / (ms_b * 1e-3)) / (total / t_seq),
            "setup_s": t_setup, "max_err_vs_sequential_normwise": d,
            "synthesis": {"ms": ms_syn, "bytes": syn_bytes, "achieved_gbs": syn_bytes / (ms_syn * 1e-3) / 1e9,
                          "peak_gbs": hbm, "frac": syn_bytes / (ms_syn * 1e-3) / 1e9 / hbm,
                          "note": f"the three batched synthesis passes timed alone (CUDA events, L2 flushed); bytes = "
                                  f"4 W + G per pair (work planes written, read and written, read; gather grid "
                                  f"written); peak = {hbm_how} HBM copy rate.  The first pass forms the "
                                  f"coefficients (Gauss-Legendre sums): it is bound by arithmetic, not bytes"}}


def run_surrogate(args, dev):
    """Learned surrogate: 5-layer BF16 MLP (tensor cores) trained on FFT-path
    samples of the remainder for (alpha, k) in [-1/2, 1/2]^2 x [1, 4]; then
    inference at near targets of many pairs with FFT-path fallback near Wood
    anomalies, against the FFT path (batched sweep) on the same targets."""
    import torch

    from paper_1801_05977_gb300 import gf
    from paper_1801_05977_gb300 import surrogate as S

    t0 = time.perf_counter()
    inp, L, _ = S.make_dataset(args.sur_train_pairs, args.sur_train_per_pair, seed=0)
    t_data = time.perf_counter() - t0
    mlp = gf.MLP(seed=0)
    t0 = time.perf_counter()
    hist = S.train(mlp, inp, L, epochs=args.sur_epochs, batch=8192, lr=2e-3, min_steps=args.sur_min_steps)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del inp, L
    # inference workload: unseen pairs (another seed), near targets
    npairs, per = args.sur_pairs, args.sur_per_pair
    # unseen pairs clear of Wood anomalies by the fallback threshold: the network serves all of them
    pr = W.sweep_pairs(npairs, seed=12345, kmin=1.0, kmax=4.0, wood_gap=1e-2)
    k, al = pr[:, 2].copy(), pr[:, :2].copy()
    x_np = np.concatenate([S.near_points(per, seed=777 + i) for i in range(npairs)])
    off = np.arange(npairs + 1, dtype=np.int64) * per
    x = torch.from_numpy(x_np).to(dev)
    times = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G, nfb = mlp.surrogate_eval(k, al, off, x, wood_delta=1e-2)
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    t_sur = float(np.mean(times))
    # the FFT path on the same targets: batched sweep (plans built, then one graph: synthesis + evaluation)
    M = np.array([S.grid_for(v) for v in k], dtype=np.int32)
    t0 = time.perf_counter()
    batch = gf.Batch(k, al, M, precision=gf.GF_FP64)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    ref = torch.empty((x.shape[0], 1), dtype=torch.complex128, device=dev)
    s = torch.cuda.Stream(device=dev)
    ft = []
    with torch.cuda.stream(s):
        for i in range(args.warmup + args.steps):
            s.synchronize()
            t0 = time.perf_counter()
            batch.run_graph(x, off, ref, gf.GF_OUT_GD, stream=s)
            s.synchronize()
            if i >= args.warmup:
                ft.append(time.perf_counter() - t0)
    t_fft = float(np.mean(ft))
    g, r = G.cpu().numpy(), ref[:, 0].cpu().numpy()

    def pair_errs(vals):
        return np.array([np.abs(vals[off[i]:off[i + 1]] - r[off[i]:off[i + 1]]).max() /
                         np.abs(r[off[i]:off[i + 1]]).max() for i in range(npairs)])

    errs = pair_errs(g)
    batch.close()
    mlp.close()
    del G

    # residual form: the network learns L_d minus a coarse plan's L_d (surrogate.COARSE
    # points per axis); at inference a coarse batched sweep of the same pairs supplies
    # that value (its plans built once: the preparation) and gf_surrogate_eval_residual
    # adds it back
    t0 = time.perf_counter()
    inp_r, L_r, _ = S.make_dataset(args.sur_train_pairs, args.sur_train_per_pair, seed=0, residual=True)
    t_data_r = time.perf_counter() - t0
    mlp_r = gf.MLP(seed=0)
    t0 = time.perf_counter()
    hist_r = S.train(mlp_r, inp_r, L_r, epochs=args.sur_epochs, batch=8192, lr=2e-3, min_steps=args.sur_min_steps)
    torch.cuda.synchronize()
    t_train_r = time.perf_counter() - t0
    del inp_r, L_r
    Mc = np.tile(np.array(S.COARSE, dtype=np.int32), (npairs, 1))
    t0 = time.perf_counter()
    cbatch = gf.Batch(k, al, Mc, precision=gf.GF_FP32_SPLIT)
    torch.cuda.synchronize()
    t_cprep = time.perf_counter() - t0
    cbase = torch.empty((x.shape[0], 1), dtype=torch.complex64, device=dev)
    rt = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cbatch.eval_points_into(x, off, cbase, gf.GF_OUT_LD)
        Gr, _ = mlp_r.surrogate_eval(k, al, off, x, wood_delta=1e-2, base=cbase[:, 0].to(torch.complex128))
        torch.cuda.synchronize()
        if i >= args.warmup:
            rt.append(time.perf_counter() - t0)
    t_res = float(np.mean(rt))
    errs_r = pair_errs(Gr.cpu().numpy())
    cbatch.close()
    mlp_r.close()
    del Gr, cbase
    # the split-precision batched FFT path (each pair's full grid) on the same targets
    sbatch = gf.Batch(k, al, M, precision=gf.GF_FP32_SPLIT)
    sref = torch.empty((x.shape[0], 1), dtype=torch.complex64, device=dev)
    st_ = []
    with torch.cuda.stream(s):
        for i in range(args.warmup + args.steps):
            s.synchronize()
            t0 = time.perf_counter()
            sbatch.run_graph(x, off, sref, gf.GF_OUT_GD, stream=s)
            s.synchronize()
            if i >= args.warmup:
                st_.append(time.perf_counter() - t0)
    t_split = float(np.mean(st_))
    errs_s = pair_errs(sref[:, 0].to(torch.complex128).cpu().numpy())
    sbatch.close()
    del sref
    residual = {"value": npairs * per / t_res, "unit": "evals/s", "s_per_call": t_res,
                "coarse_grid": "x".join(map(str, S.COARSE)), "coarse_plans_setup_s": t_cprep,
                "value_with_setup": npairs * per / (t_res + t_cprep),
                "err_vs_fft_path_normwise": {"median": float(np.median(errs_r)),
                                             "p90": float(np.percentile(errs_r, 90)), "max": float(errs_r.max())},
                "training": {"samples": args.sur_train_pairs * args.sur_train_per_pair, "epochs": len(hist_r),
                             "final_loss": hist_r[-1], "train_s": t_train_r, "data_s": t_data_r},
                "how": "per call: coarse batched sweep (split) GF_OUT_LD at the targets + gf_surrogate_eval_residual"}
    split_path = {"value": npairs * per / t_split, "unit": "evals/s", "s_per_call": t_split,
                  "err_vs_fft_path_normwise": {"median": float(np.median(errs_s)), "max": float(errs_s.max())},
                  "how": "split-precision batched sweep (graph: synthesis + evaluation) of each pair's full grid"}
    # tensor-core GEMM of one hidden layer at inference size: (2^20 x 256) . (256 x 256)^T
    A = torch.randn((1 << 20, 256), device=dev).to(torch.bfloat16)
    Bm = torch.randn((256, 256), device=dev).to(torch.bfloat16)
    gt = []
    for i in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gf.gemm_bf16(A, Bm)
        e1.record()
        torch.cuda.synchronize()
        if i >= 2:
            gt.append(e0.elapsed_time(e1))
    gemm_ms = float(np.mean(gt))
    gemm_tf = 2.0 * (1 << 20) * 256 * 256 / (gemm_ms * 1e-3) / 1e12
    # fused network forward (all layers on chip) on 2^20 samples
    mlp2 = gf.MLP(seed=1)
    xin = torch.rand((1 << 20, 6), device=dev)
    ft2 = []
    for i in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mlp2.forward(xin)
        e1.record()
        torch.cuda.synchronize()
        if i >= 2:
            ft2.append(e0.elapsed_time(e1))
    mlp2.close()
    fwd_ms = float(np.mean(ft2))
    fwd_flops = 2.0 * (80 * 256 + 3 * 256 * 256 + 256 * 2) * (1 << 20)
    bf16_peak, bf16_how = measured_peak("bf16_tflops", 1900.0)
    total = npairs * per
    return {"value": total / t_sur, "unit": "evals/s", "s_per_call": t_sur, "pairs": npairs,
            "gemm_bf16": {"shape": "M=2^20, N=256, K=256 (per-layer kernel, fp32 out)", "ms": gemm_ms,
                          "tflops": gemm_tf},
            "fused_forward": {"samples": 1 << 20, "ms": fwd_ms, "tflops": fwd_flops / (fwd_ms * 1e-3) / 1e12,
                              "frac_of_bf16_peak": fwd_flops / (fwd_ms * 1e-3) / 1e12 / bf16_peak,
                              "peak": f"{bf16_peak} TFLOP/s bf16 ({bf16_how}, burst)"},
            "targets_per_pair": per, "targets": "near region |x3| <= c", "dtype": "bf16 weights, fp32 accumulation",
            "fallback_pairs": nfb, "wood_delta": 1e-2,
            "fft_path": {"value": total / t_fft, "s_per_call": t_fft, "setup_s": t_setup,
                         "how": "batched sweep (graph) of FP64 plans on the same targets; setup excluded"},
            "speedup_vs_fft_path": t_fft / t_sur,
            "speedup_vs_fft_path_with_setup": (t_fft + t_setup) / t_sur,
            "err_vs_fft_path_normwise": {"median": float(np.median(errs)), "p90": float(np.percentile(errs, 90)),
                                         "max": float(errs.max())},
            "training": {"samples": args.sur_train_pairs * args.sur_train_per_pair, "epochs": len(hist),
                         "batch": 8192, "final_loss": hist[-1], "train_s": t_train, "data_s": t_data},
            "residual": residual, "split_fft_path": split_path}


def run_configs(args, dev, flush):
    """The other configurations, one plan + evaluation per step (device time):
    2D G (k = 1.3, alpha = 0.2, 64 x 64, 1e4 targets, complex128), the 2D
    derivatives of Sec. 2.4 (gradient and second-derivative differences, 256 x 256)
    and the Maxwell
    tensor (k = 2.5, alpha = (0.1, 0.3), 256 x 256 x 64, six entries, float bulk
    with double singular part; 1e6 targets, 10% clustered within 0.05 of lattice
    points; its error stated against the double-precision path on the GPU)."""
    import torch

    from paper_1801_05977_gb300 import gf

    def timed(mk, x, which, steps, warm, out):
        ts, ph = [], []
        for i in range(warm + steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            p = mk()
            p.eval_points_into(x, out, which)
            e1.record()
            torch.cuda.synchronize()
            if i >= warm:
                ts.append(e0.elapsed_time(e1))
                ph.append(p.phase_ms())
            p.close()
        return float(np.mean(ts)), ph

    res = {}
    x2 = torch.from_numpy(W.targets_2d(10_000, seed=0)).to(dev)
    o2 = torch.empty((10_000, 1), dtype=torch.complex128, device=dev)
    ms, ph = timed(lambda: gf.Plan(2, 1.3, (0.2,), (64, 64)), x2, gf.GF_OUT_G, args.steps, args.warmup, o2)
    res["2d_G"] = {"workload": "2D quasi-periodic G, k=1.3, alpha=0.2, grid 64x64, 1e4 uniform targets",
                   "value": 1e4 / (ms * 1e-3), "unit": "evals/s", "ms_per_step": ms, "dtype": "f64",
                   "phases_ms": {"synthesis": float(np.mean([p[0] for p in ph])), "near": float(np.mean([p[2] for p in ph])),
                                 "far": float(np.mean([p[3] for p in ph]))}}
    # 2D derivatives (Sec. 2.4): one derivative plan (L, K_1 - h_1, K_2 - h_2 and the
    # three T_pq - h_pq fields for k2) and both outputs per step
    nd = 100_000
    xd = torch.from_numpy(W.targets_2d(nd, seed=1)).to(dev)
    og, oh = (torch.empty((nd, 3), dtype=torch.complex128, device=dev) for _ in range(2))
    ts, ph = [], []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        p = gf.Plan(2, 1.3, (0.2,), (256, 256), kind=gf.GF_DERIV2D, k2=2.1, c_tilde=1.4)
        p.eval_points_into(xd, og, gf.GF_OUT_GRAD)
        p.eval_points_into(xd, oh, gf.GF_OUT_HESSDIFF)
        e1.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            ts.append(e0.elapsed_time(e1))
            ph.append(p.phase_ms())
        p.close()
    msd = float(np.mean(ts))
    res["2d_deriv"] = {"workload": "2D derivatives (Sec. 2.4): G, dG/dx1, dG/dx2 and T11, T12, T22 for k=1.3, "
                                   "k2=2.1, alpha=0.2, c~=1.4, grid 256x256 (6 fields), 1e5 uniform targets",
                       "value": nd / (msd * 1e-3), "unit": "targets/s (6 entries each: both outputs)",
                       "ms_per_step": msd, "dtype": "f64",
                       "synthesis_ms": float(np.mean([q[0] for q in ph]))}
    x3 = torch.from_numpy(W.targets_3d_clustered(1_000_000, seed=0)).to(dev)
    o32 = torch.empty((1_000_000, 6), dtype=torch.complex64, device=dev)
    ms32, ph32 = timed(lambda: gf.Plan(3, 2.5, (0.1, 0.3), (256, 256, 64), precision=gf.GF_FP32_SPLIT,
                                       kind=gf.GF_MAXWELL), x3, gf.GF_OUT_MAXWELL6, args.steps, args.warmup, o32)
    o64 = torch.empty((1_000_000, 6), dtype=torch.complex128, device=dev)
    ms64, ph64 = timed(lambda: gf.Plan(3, 2.5, (0.1, 0.3), (256, 256, 64), kind=gf.GF_MAXWELL), x3,
                       gf.GF_OUT_MAXWELL6, 1, 1, o64)
    d = (o32.to(torch.complex128) - o64).abs()
    err = float((d.max(dim=0).values / o64.abs().max(dim=0).values).max())
    res["maxwell"] = {"workload": "Maxwell tensor (6 entries), k=2.5, alpha=(0.1,0.3), grid 256x256x64, 1e6 targets, "
                                  "10% clustered within 0.05 of lattice points",
                      "value": 1e6 / (ms32 * 1e-3), "unit": "evals/s (tensor = 6 entries)", "ms_per_step": ms32,
                      "dtype": "f32/f64 split", "max_entry_err_vs_fp64_normwise": err,
                      "phases_ms": {"synthesis": float(np.mean([p[0] for p in ph32])),
                                    "near": float(np.mean([p[2] for p in ph32])),
                                    "far": float(np.mean([p[3] for p in ph32]))},
                      "fp64": {"value": 1e6 / (ms64 * 1e-3), "ms_per_step": ms64,
                               "phases_ms": {"synthesis": ph64[0][0], "near": ph64[0][2], "far": ph64[0][3]}}}
    return res


def run_batch_only(args):
    """Profiling helper: the batched-sweep leg alone (plans, autotune, graph
    steps and the pair-after-pair comparison), its result line printed."""
    import torch

    dev = torch.device("cuda", 0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    print(json.dumps({"batched": run_batched(args, dev, flush)}))
    return 0


def run_mlp_forward(args):
    """Profiling helper: fused forward passes of the surrogate network on
    `mlp_forward_only` random samples (two, then `steps` timed by CUDA events);
    prints their mean time and rate."""
    import torch

    from paper_1801_05977_gb300 import gf

    mlp = gf.MLP(seed=1)
    x = torch.rand((args.mlp_forward_only, 6), device="cuda")
    for _ in range(2):
        mlp.forward(x)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mlp.forward(x)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    mlp.close()
    ms = float(np.mean(ts))
    flops = 2.0 * (80 * 256 + 3 * 256 * 256 + 256 * 2) * args.mlp_forward_only
    print(json.dumps({"mlp_forward": {"samples": args.mlp_forward_only, "ms": ms, "tflops": flops / (ms * 1e-3) / 1e12,
                                      "note": "per call of gf.MLP.forward (features, fused network, output)"}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gf", choices=["gf", "reference"])
    ap.add_argument("--ref-sample", type=int, default=50000,
                    help="targets per step of the reference arm (the oracle), beside the full plan")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--targets", type=int, default=N_TARGETS,
                    help="targets per step (the benchmark workload is 1e6; smaller only for profiling captures)")
    ap.add_argument("--paths", default="both", choices=["both", "fp64", "split", "split_far_grid"],
                    help="which precision paths to run (profiling captures run one)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling captures)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-sweep leg")
    ap.add_argument("--batch-pairs", type=int, default=256)
    ap.add_argument("--batch-targets", type=int, default=100_000)
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-surrogate leg")
    ap.add_argument("--no-configs", action="store_true", help="skip the 2D and Maxwell configurations")
    ap.add_argument("--mlp-forward-only", type=int, default=0, help="profiling: only run the fused network forward")
    ap.add_argument("--batch-only", action="store_true", help="profiling: only run the batched-sweep leg")
    ap.add_argument("--sur-train-pairs", type=int, default=1000)
    ap.add_argument("--sur-train-per-pair", type=int, default=10_000)
    ap.add_argument("--sur-epochs", type=int, default=2)
    ap.add_argument("--sur-min-steps", type=int, default=8000)
    ap.add_argument("--sur-pairs", type=int, default=1000)
    ap.add_argument("--sur-per-pair", type=int, default=10_000)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mlp_forward_only:
        return run_mlp_forward(args)
    if args.batch_only:
        return run_batch_only(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
