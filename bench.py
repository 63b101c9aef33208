#!/usr/bin/env python
"""Benchmark: MINRES solves/s at true relative residual 1e-8 for the
complex-shifted Laplacian solve (K + lambda I) z = f with the absolute-value
preconditioner (arXiv 2408.00488), on the 2D n=1023 workload:
a(x, y) = exp(ln(10) x y), lambda = 100i, f ~ U[-1,1] + i U[-1,1] (seed 1).

A step is one whole solve (ingest, P^{-1} b, the MINRES loop with its
stopping test, egress) with f already resident in HBM.  The headline `value`
is the FP32-preconditioner form (sine transforms and scale of P^{-1} in FP32;
stencil, Lanczos, Givens and residual norms in FP64); the plain FP64 form is
timed beside it under "forms".  Both must reach relres <= 1e-8.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl csl|reference]
Multi-GPU (torchrun, one rank per GPU): independent replicas of the solve
("replicas only": the method has no exchange step), value = total solves/s.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MINRES solves/s at relres 1e-8 (2D n=1023, a=exp(ln10*x*y), lambda=100i)"
UNIT = "solves/s"
WORKLOAD = ("config1: 2D unit square, n=1023 (M=1,046,529), 5-point FD of -div(a grad), "
            "a=exp(ln10*x*y) at face midpoints, lambda=0+100i, f~U[-1,1]^2 seed 1, tol 1e-8")
TOL = 1e-8
MAXIT = 2000
HEADLINE_ARITH = ("MINRES with FP32 sine transforms and per-mode scale inside P^-1; the stencil, the Lanczos "
                  "vectors and step and the w/x update in float-pair (double-float, about 2^-47) arithmetic; "
                  "Lanczos/Givens scalars, reductions and the true-residual check in FP64 (a further variant of "
                  "the FP32-preconditioner form; the form with FP64 vectors is forms.fp32_precond)")


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 / FP32 ALU peaks derived from unit counts and the maximum SM clock:
# 152 SMs x 2 FP64 FMA/clk (x 2 flops) x 2.07 GHz, and 152 x 128 FP32 FMA/clk.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def kernel_source_hash():
    """Hash of the CUDA sources: a committed ncu traffic figure is used only
    while the kernels are unchanged since it was captured."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2408_00488_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        if fn.endswith((".cu", ".cuh")):
            with open(os.path.join(d, fn), "rb") as fh:
                h.update(fn.encode())
                h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel_name, prec):
    """DRAM bytes per launch of `kernel_name` (FP32/FP64 form of this
    workload) from profiles/traffic.json, or None when absent or stale."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get("kernels", {}).get(prec, {}).get(kernel_name)


def golden_iters(name):
    p = os.path.join(ROOT, "tests", "golden", "oracle_iterations.txt")
    try:
        with open(p) as fh:
            for line in fh:
                if line.startswith(name + " "):
                    return int(line.split()[1])
    except OSError:
        pass
    return None


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def kernel_model(name, M, d, prec, N, ff=False):
    """Algorithmic bytes and flops per launch of one kernel of a MINRES
    iteration (M grid points, d dims, line length N = n+1 of the pass axis).
    prec: "fp64", "fp32" (FP32 transforms, float-pair vectors) or
    "fp32_precond" (FP32 transforms, FP64 vectors and stencil).
    ff: the stencil runs in float-pair arithmetic (faces as 8-byte pairs, no
    diagonal; its FP32 instructions counted as 2 flops each, so that they
    meet the FP32 peak at the instruction issue rate)."""
    if prec == "fp32_precond":  # the FP64 form's vector work around FP32 transforms
        b64, f64_, f32_ = kernel_model(name, M, d, "fp64", N)
        b32, f64t, f32t = kernel_model(name, M, d, "fp32", N)
        if name == "k_stencil":
            return b64 - 8 * M, f64_, 0.0  # z read as FP32
        if name.startswith("k_row<LOAD_LANCZOS"):
            return b64 - 8 * M, 4.0 * M, f32t - 2 * 36 * M
        if name == "k_update":
            return b64 - 8 * M, f64_, 0.0
        return b32, f64t, f32t
    sT = 16 if prec == "fp64" else 8
    dst_flops = 11 + 5 * math.log2(N)  # per complex point per sine transform (pre, FFT, split, scan)
    f64 = f32 = 0.0
    if name == "k_stencil" and ff:
        b = sT + 16 + 16 + 8 * d
        f32 = 2 * (74 + 72 * d)  # pair arithmetic: alpha, 2d fluxes, beta, delta and u' terms, 2 components
    elif name == "k_stencil":
        b = sT + 16 + 16 + 8 + 8 * d
        f64 = 16 + 8 * d
    elif name.startswith("k_row<LOAD_LANCZOS"):
        b = 16 + 16 + 16 + sT
        if prec == "fp64":
            f64 = 4 + dst_flops
        else:
            f32 = 2 * 36 + dst_flops  # the Lanczos step in float pairs
    elif name.startswith("k_row<LOAD_T,STORE_Z_UPDATE"):
        b = sT + sT + 48 + sT + 32
        f64 = 14
        if prec == "fp64":
            f64 += dst_flops
        else:
            f32 += dst_flops
    elif name.startswith("k_row<LOAD_T,STORE_Z>"):  # inverse x transform only (update split off)
        b = 2 * sT
        if prec == "fp64":
            f64 += dst_flops
        else:
            f32 += dst_flops
    elif name == "k_update":  # w_{j+1}, x_j: z_j, w_{j-1}, w_j, x in; w_{j+1}, x out
        b = sT + 80
        if prec == "fp64":
            f64 = 12
        else:
            f32 = 2 * 96  # float pairs
    elif name == "k_strided<mid>":
        b = 2 * sT + (8 if prec == "fp64" else 0)
        fl = 2 * dst_flops + 7
        if prec == "fp64":
            f64 += fl
        else:
            f32 += fl
    else:  # plain strided transform (3D y passes)
        b = 2 * sT
        if prec == "fp64":
            f64 += dst_flops
        else:
            f32 += dst_flops
    return b * M, f64 * M, f32 * M


def roofline_table(kernels, M, d, prec, n, hbm_gbs, iters, ff=False):
    out = []
    per_iter_ms = sum(ms for _, ms in kernels)
    for name, ms in kernels:
        N = n + 1
        B, F64, F32 = kernel_model(name, M, d, prec, N, ff)
        s = ms / 1e3
        t_hbm = B / (hbm_gbs * 1e9)
        t64 = F64 / (FP64_PEAK_TFLOPS * 1e12)
        t32 = F32 / (FP32_PEAK_TFLOPS * 1e12)
        if t64 >= max(t_hbm, t32):
            bound, achieved, peak, unit = "alu", F64 / s / 1e12, FP64_PEAK_TFLOPS, "TFLOP/s"
        elif t32 > t_hbm:
            bound, achieved, peak, unit = "alu", F32 / s / 1e12, FP32_PEAK_TFLOPS, "TFLOP/s"
        else:
            bound, achieved, peak, unit = "hbm", B / s / 1e9, hbm_gbs, "GB/s"
        out.append({"kernel": name, "ms": round(ms, 5), "share": round(ms / per_iter_ms, 4),
                    "alg_bytes": int(B), "fp64_flops": int(F64), "fp32_flops": int(F32),
                    "hbm_gbs": round(B / s / 1e9, 1), "hbm_frac": round(B / s / 1e9 / hbm_gbs, 4),
                    "fp64_tflops": round(F64 / s / 1e12, 4),
                    "bound": bound, "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": unit,
                    "frac": round(achieved / peak, 4)})
    return out


# ---------------------------------------------------------------------------
ORACLE_SAMPLE_ITERS = 40


def oracle_seconds_per_iteration(k=ORACLE_SAMPLE_ITERS):
    """One bounded sample of the FP64 CPU oracle on the workload: the first k
    MINRES iterations of its solve (set-up included, as in a full solve);
    returns (seconds per iteration, iterations run)."""
    import oracle
    import workloads as W

    s = W.config1()
    t = time.perf_counter()
    _, info = oracle.solve(s.faces, s.lam, s.f, tol=1e-300, maxit=k)
    dt = time.perf_counter() - t
    return dt / info.iters, info.iters


def cpu_oracle_sample():
    """The cpu_baseline leg: the same 40-iteration sample as the reference arm."""
    return oracle_seconds_per_iteration(ORACLE_SAMPLE_ITERS)


def run_reference(args, rank, world):
    """The oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    import workloads as W

    iters_full = golden_iters("config1")
    k_per_step = ORACLE_SAMPLE_ITERS
    times = []
    for i in range(args.warmup + args.steps):
        per, _ = oracle_seconds_per_iteration(k_per_step)
        if i >= args.warmup:
            times.append(per)
    per_iter = statistics.mean(times)
    value = 1.0 / (per_iter * iters_full) if iters_full else None
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_iter * k_per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step = the first {k_per_step} MINRES iterations of the workload's "
                                       f"solve, set-up included (oracle.solve, FP64 NumPy, dense O(n^2) DST-I, "
                                       f"explicit residual per iteration); solves/s = 1 / (s per iteration x "
                                       f"{iters_full} iterations of the full oracle solve); the same sample as "
                                       f"the cpu_baseline of the GPU arm"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile(name):
    import numpy as np
    import torch

    import workloads as W
    import paper_2408_00488_gb300 as csl

    s = getattr(W, name)()
    faces = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in s.faces]
    f = torch.from_numpy(np.ascontiguousarray(s.f)).cuda()
    for prec in (("fp32", "fp32_precond", "fp64") if name == "config1" else ("bf16x6", "bf16x3", "fp32")):
        with csl.Plan(faces, s.lam, precision=prec) as plan:
            plan.solve(f, tol=TOL, maxit=MAXIT)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("prof")
            kt = plan.time_kernels(1)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            print(name, prec, plan.config, [(k, round(ms * 1e3, 1)) for k, ms in kt], flush=True)


# ---- replicas (one process per GPU; no data-path collective) ---------------
def init_replicas(backend):
    """Rank, world size, local rank and the torch.distributed module (None for
    a single process) from the torchrun environment; one GPU per rank."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
    return rank, world, local_rank, dist


def replica_max(x, dist, device="cpu"):
    """The slowest replica's time: maximum of a per-rank float over all ranks."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_max):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank * 1e3 / ms_max


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="csl", choices=["csl", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel-reps", type=int, default=20)
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven iteration loop (every kernel a separate launch, for launch lists)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched config-3 line")
    ap.add_argument("--no-config2", action="store_true", help="skip the config-2 forms (FFT vs tensor-core DST)")
    ap.add_argument("--no-paradiag", action="store_true", help="skip the all-at-once time-solve line")
    ap.add_argument("--no-tables", action="store_true", help="skip the paper's table rows at n = 1023, 4095, 16383")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file: loaded before the plans are made when it exists, "
                         "written after them, so that a later (e.g. profiled) run takes the same shapes")
    ap.add_argument("--profile", choices=["config1", "config2"], default=None,
                    help="solve once, then launch each kernel of one MINRES iteration inside an "
                         "NVTX range 'prof' for an ncu capture (--nvtx --nvtx-include prof/); config1: fp32, "
                         "fp32_precond and fp64 forms, config2: bf16x6, bf16x3 and fp32; no JSON")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank, world, local_rank, dist = init_replicas("nccl")

    if args.tune_cache and args.impl == "csl":
        import paper_2408_00488_gb300 as csl
        if os.path.exists(args.tune_cache):
            csl.tune_cache_load(args.tune_cache)
    if args.profile:
        run_profile(args.profile)
        if args.tune_cache:
            csl.tune_cache_save(args.tune_cache)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    import numpy as np
    import torch

    import workloads as W
    import paper_2408_00488_gb300 as csl

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    s = W.config1()
    n, d, M = s.n, s.dim, s.M
    faces = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in s.faces]
    f = torch.from_numpy(np.ascontiguousarray(s.f)).to(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MiB)
    hbm_gbs, hbm_src = read_peaks()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, K, tag):
        """K steps, each bracketed by CUDA events on the current stream, L2
        flushed (outside the events) before every step; returns mean ms.  The
        steps sit in the NVTX range `tag` (for ncu --nvtx-include "tag/")."""
        ms = []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(tag)
        for _ in range(K):
            flush.zero_()
            e0.record()
            info = fn()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        torch.cuda.nvtx.range_pop()
        return statistics.mean(ms), info

    def max_over_ranks(x):
        return replica_max(x, dist, dev)

    forms = {}
    plans = {}
    for prec in ("fp32", "fp32_precond", "fp64"):
        plans[prec] = csl.Plan(faces, s.lam, precision=prec, use_graph=not args.no_graph)
        z = torch.empty_like(f)
        for _ in range(args.warmup):
            _, info = plans[prec].solve(f, tol=TOL, maxit=MAXIT, out=z)
        assert info.converged and info.relres <= TOL, (prec, info)
    if args.tune_cache:
        csl.tune_cache_save(args.tune_cache)

    gpu_id = "0"
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local_rank)
    sampler = ClockSampler(gpu_id)

    # ---- timed region: headline form (FP32 preconditioner) -------------------
    z = torch.empty_like(f)
    barrier()
    sampler.start()
    ms_mixed, info_mixed = timed(lambda: plans["fp32"].solve(f, tol=TOL, maxit=MAXIT, out=z)[1], args.steps, "timed_fp32")
    barrier()
    clocks = sampler.stop()
    ms_mixed = max_over_ranks(ms_mixed)
    assert info_mixed.converged and info_mixed.relres <= TOL
    forms["fp32_pairs"] = {"solves_per_s": job_rate(1, world, ms_mixed), "ms_per_solve": ms_mixed,
                           "iters": info_mixed.iters, "oracle_iters": golden_iters("config1"),
                           "relres": info_mixed.relres, "launches_per_solve": info_mixed.launches,
                           "arithmetic": HEADLINE_ARITH}

    # ---- FP32 only inside P^-1, every vector and the stencil in FP64 --------
    barrier()
    ms_sp, info_sp = timed(lambda: plans["fp32_precond"].solve(f, tol=TOL, maxit=MAXIT, out=z)[1], args.steps,
                           "timed_fp32_precond")
    barrier()
    ms_sp = max_over_ranks(ms_sp)
    assert info_sp.converged and info_sp.relres <= TOL
    forms["fp32_precond"] = {"solves_per_s": job_rate(1, world, ms_sp), "ms_per_solve": ms_sp,
                             "iters": info_sp.iters, "oracle_iters": golden_iters("config1"),
                             "relres": info_sp.relres, "launches_per_solve": info_sp.launches,
                             "arithmetic": "FP32 sine transforms and per-mode scale inside P^-1; stencil, "
                                           "Lanczos vectors and step, w/x update, Givens, reductions and "
                                           "residual check in FP64"}

    # ---- plain FP64 form ---------------------------------------------------
    barrier()
    ms_64, info_64 = timed(lambda: plans["fp64"].solve(f, tol=TOL, maxit=MAXIT, out=z)[1], args.steps, "timed_fp64")
    barrier()
    ms_64 = max_over_ranks(ms_64)
    assert info_64.converged and info_64.relres <= TOL
    forms["fp64"] = {"solves_per_s": job_rate(1, world, ms_64), "ms_per_solve": ms_64, "iters": info_64.iters,
                     "oracle_iters": golden_iters("config1"), "relres": info_64.relres,
                     "launches_per_solve": info_64.launches, "arithmetic": "FP64 throughout (the paper's)"}

    # ---- end to end through the C ABI with host buffers (pinned) -------------
    fh = torch.from_numpy(np.ascontiguousarray(s.f)).pin_memory()
    zh = torch.empty_like(fh).pin_memory()
    for _ in range(2):
        plans["fp32"].solve_host(fh, zh, tol=TOL, maxit=MAXIT)
    barrier()
    ms_e2e, info_e2e = timed(lambda: plans["fp32"].solve_host(fh, zh, tol=TOL, maxit=MAXIT), args.steps, "timed_e2e")
    barrier()
    ms_e2e = max_over_ranks(ms_e2e)
    assert info_e2e.converged

    # ---- per-kernel durations (CUDA events on the launching stream) --------
    kern = {}
    for prec, key in (("fp32", "fp32_pairs"), ("fp32_precond", "fp32_precond"), ("fp64", "fp64")):
        p = plans[prec]
        p.solve(f, tol=TOL, maxit=MAXIT, out=z)  # real data in the vectors
        kt = p.time_kernels(args.kernel_reps)
        kern[key] = roofline_table(kt, M, d, prec, n, hbm_gbs, forms[key]["iters"],
                                   ff="stencil[float-pair" in p.config)
    head = kern["fp32_pairs"]
    dom = max(head, key=lambda r: r["ms"])
    roofline = {"kernel": dom["kernel"], "bound": dom["bound"], "achieved": dom["achieved"],
                "peak": dom["peak"], "unit": dom["unit"], "frac": dom["frac"],
                "traffic": committed_traffic(dom["kernel"], "fp32"),
                "peak_source": (f"HBM {hbm_src} (MEASURED_PEAKS.json)" if dom["bound"] == "hbm" else
                                "derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz (probe measured 1.196 TFLOP/s)"
                                if dom["peak"] == round(FP64_PEAK_TFLOPS, 4) else
                                "derived: 152 SMs x 128 FP32 FMA/clk x 2.07 GHz")}
    # whole-solve HBM fraction of the headline form: algorithmic bytes per iteration
    bytes_iter = sum(r["alg_bytes"] for r in head)
    solve_bytes = bytes_iter * info_mixed.iters
    hbm_pct_solve = solve_bytes / (ms_mixed / 1e3) / (hbm_gbs * 1e9)

    # ---- batched shifts (config 3): 192 systems in one graph launch ---------
    batched = None
    if not args.no_batch:
        systems = W.config3()
        dfaces = {}
        for sy in systems:
            if id(sy.faces) not in dfaces:
                dfaces[id(sy.faces)] = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in sy.faces]
        fs = [torch.from_numpy(np.ascontiguousarray(sy.f)).to(dev) for sy in systems]
        batched = {"workload": "config3: 2D n in {127,255,511} x 64 alpha-circulant shifts (L=64, eps=1e-4), "
                               "a = 1+0.5 sin(pi x) sin(pi y), f ~ U[-1,1]^2 seed 3; 192 systems per step"}
        for prec in ("fp32", "bf16x6", "fp64"):
            B = csl.Batch([(dfaces[id(sy.faces)], sy.lam) for sy in systems], precision=prec)
            for _ in range(2):
                B.solve(fs, tol=TOL, maxit=MAXIT)
            barrier()
            msb, infos = timed(lambda: B.solve(fs, tol=TOL, maxit=MAXIT)[1], max(2, args.steps // 2), "timed_batch_" + prec)
            barrier()
            msb = max_over_ranks(msb)
            assert all(i.converged and i.relres <= TOL for i in infos)
            its = [i.iters for i in infos]
            batched[prec] = {"solves_per_s": job_rate(len(systems), world, msb), "ms_per_batch": msb,
                             "iters_min": min(its), "iters_max": max(its),
                             "max_relres": max(i.relres for i in infos)}
            B.close()
        # one synchronisation point between dependent stages: a kernel
        # boundary of the batch's graph (PDL) against a grid barrier of one
        # persistent cooperative kernel
        batched["sync_cost_us"] = {k: round(v, 3) for k, v in csl.probe_sync_cost().items()}

    # ---- config 2 (3D n = 127): FFT vs split-BF16 tensor-core transforms ---
    cfg2 = None
    if not args.no_config2:
        s2 = W.config2()
        faces2 = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in s2.faces]
        f2 = torch.from_numpy(np.ascontiguousarray(s2.f)).to(dev)
        z2 = torch.empty_like(f2)
        cfg2 = {"workload": "config2: 3D n=127 (M=2,048,383), a = 1+0.9 sin2pix sin2piy sin2piz at face midpoints, "
                            "lambda=-5+50i, f ~ N(0,1)^2 seed 2, tol 1e-8"}
        for prec in ("fp64", "fp32", "bf16x3", "bf16x6"):
            p2 = csl.Plan(faces2, s2.lam, precision=prec)
            for _ in range(2):
                p2.solve(f2, tol=TOL, maxit=MAXIT, out=z2)
            barrier()
            ms2, inf2 = timed(lambda: p2.solve(f2, tol=TOL, maxit=MAXIT, out=z2)[1], max(3, args.steps // 2),
                              "timed_c2_" + prec)
            barrier()
            ms2 = max_over_ranks(ms2)
            assert inf2.converged and inf2.relres <= TOL
            kt = p2.time_kernels(args.kernel_reps)
            cfg2[prec] = {"solves_per_s": job_rate(1, world, ms2), "ms_per_solve": ms2, "iters": inf2.iters,
                          "relres": inf2.relres, "us_per_iter": ms2 * 1e3 / inf2.iters,
                          "kernels_us": {k: round(ms * 1e3, 1) for k, ms in kt}, "plan": p2.config}
            p2.close()

    # ---- all-at-once backward Euler (csl_paradiag): the config-3 setting ----
    pdline = None
    if not args.no_paradiag:
        n3, L3, a3 = 127, 64, 1e-4
        tau3 = 1.0 / L3
        fc3 = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in W.sample_faces(2, n3, W.coef_c0)]
        u0 = torch.from_numpy(W.rhs_uniform((n3, n3), 62)).to(dev)
        g3 = torch.from_numpy(W.rhs_normal((L3, n3, n3), 63) * 0.1).to(dev)
        pd = csl.ParaDiag(fc3, L3, tau3, a3, precision="fp32")
        for _ in range(2):
            pd.solve(u0, g3, tol=1e-10, maxit=10, inner_tol=1e-10)
        barrier()
        ms_pd, pinfo = timed(lambda: pd.solve(u0, g3, tol=1e-10, maxit=10, inner_tol=1e-10)[1],
                             max(3, args.steps // 2), "timed_paradiag")
        barrier()
        ms_pd = max_over_ranks(ms_pd)
        assert pinfo.status == 0 and pinfo.relres <= 1e-10
        pd.close()
        # one implicit step (K + I/tau) u = rhs at the same accuracy: L of them,
        # one after the other, are what sequential time stepping costs
        ps = csl.Plan(fc3, 1.0 / tau3, precision="fp32")
        rhs = g3[0].contiguous()
        for _ in range(2):
            ps.solve(rhs, tol=1e-10, maxit=MAXIT)
        ms_step, sinfo = timed(lambda: ps.solve(rhs, tol=1e-10, maxit=MAXIT)[1], max(3, args.steps // 2),
                               "timed_step")
        ps.close()
        pdline = {"workload": f"backward Euler u' + K u = g on [0,1], 2D n={n3} (a as config 0), L={L3} steps, "
                              f"alpha-circulant a={a3}; u0 ~ U[-1,1]^2 seed 62, g ~ 0.1 N(0,1)^2 seed 63; "
                              f"tol 1e-10 on the all-at-once residual",
                  "ms_per_solve": ms_pd, "time_steps_per_s": job_rate(L3, world, ms_pd), "sweeps": pinfo.sweeps,
                  "relres": pinfo.relres, "inner_iters_max": pinfo.inner_iters_max,
                  "sequential_estimate_ms": L3 * ms_step, "step_iters": sinfo.iters,
                  "speedup_vs_sequential": L3 * ms_step / ms_pd}

    # ---- the paper's Tables 1(a) / 2(a) rows (FP64 form, as the paper) -----
    # CPU seconds the paper prints (Table 1(a): a = 1; Table 2(a): a =
    # (20+x^2)(20+y^2); Octave on 2x Xeon Gold 6246R), context only
    paper_s = {("1a", 1023): [0.89, 0.82, 0.83, 0.83, 0.99, 0.93],
               ("1a", 4095): [20.65, 22.71, 20.71, 20.55, 23.22, 23.09],
               ("1a", 16383): [322.73, 335.83, 356.19, 334.66, 353.76, 355.89],
               ("2a", 1023): [4.59, 4.67, 4.14, 4.47, 4.13, 4.34],
               ("2a", 4095): [114.74, 114.66, 110.62, 109.70, 111.25, 110.60],
               ("2a", 16383): [1670.2, 1666.5, 1680.3, 1683.6, 1715.0, 1777.1]}
    tables = None
    if not args.no_tables:
        tables = {"workload": "Tables 1(a)/2(a) rows: 2D n in {1023, 4095, 16383}, a = 1 (1a) or (20+x^2)(20+y^2) "
                              "(2a), the paper's six (alpha, beta) per table (the first one at n = 16383), "
                              "f ~ N(0,1)^2 seed 81, tol 1e-8, FP64 form; "
                              "ms = one solve (plan set-up excluded, as the paper's timings are per solve)",
                  "rows": []}
        for (tab, nt), cpu_s in paper_s.items():
            coef = W.coef_const(1.0) if tab == "1a" else W.coef_table2
            shifts = W.TABLE1_SHIFTS if tab == "1a" else W.TABLE2_SHIFTS
            ft = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in W.sample_faces(2, nt, coef)]
            fr = torch.from_numpy(W.rhs_normal((nt, nt), 81)).to(dev)
            zt = torch.empty_like(fr)
            rows_here = list(zip(shifts, cpu_s))
            if nt > 4095:  # the largest grid: one shift per table keeps the bench within minutes
                rows_here = rows_here[:1]
            for (al, be), cs in rows_here:
                with csl.Plan(ft, al + 1j * be, precision="fp64") as pt:
                    pt.solve(fr, tol=TOL, maxit=MAXIT, out=zt)
                    ms_t, it_t = timed(lambda: pt.solve(fr, tol=TOL, maxit=MAXIT, out=zt)[1], 3,
                                       f"timed_table_{tab}_{nt}")
                assert it_t.converged
                tables["rows"].append({"table": tab, "n": nt, "alpha": al, "beta": be, "iters": it_t.iters,
                                       "ms": round(ms_t, 3), "paper_iters": 2 if tab == "1a" else 14,
                                       "paper_cpu_s": cs, "ratio_vs_paper_cpu": round(cs * 1e3 / ms_t, 1)})
            del ft, fr, zt

    # ---- CPU baseline: the oracle on a bounded sample ----------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per_iter, k = cpu_oracle_sample()
        it_full = golden_iters("config1") or info_64.iters
        cpu = {"value": 1.0 / (per_iter * it_full), "unit": UNIT, "cores": len(os.sched_getaffinity(0)),
               "kind": "oracle",
               "sample": f"{k} MINRES iterations of this workload's solve by oracle.solve (FP64 NumPy, "
                         f"dense O(n^2) DST-I, explicit residual per iteration); solves/s = 1/(s per iteration "
                         f"x {it_full} iterations of the full oracle solve)"}

    if rank == 0:
        bytes_io = 16 * M
        line = {
            "metric": METRIC, "value": job_rate(1, world, ms_mixed), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inside P^-1; f32x2 float-pair vectors and stencil; f64 scalars and residual check",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": HEADLINE_ARITH,
                       "l2": "flushed (256 MiB write) before every step", "parallelism": "replicas" if world > 1
                       else "single GPU"},
            "forms": forms,
            "roofline": roofline,
            "solve_hbm_frac": round(hbm_pct_solve, 4),
            "batched": batched,
            "config2_forms": cfg2,
            "paradiag": pdline,
            "paper_tables": tables,
            "plan_config": {k: plans[p].config for k, p in (("fp32_pairs", "fp32"), ("fp32_precond", "fp32_precond"),
                                                             ("fp64", "fp64"))},
            "kernels": kern,
            "cpu_baseline": cpu,
            "e2e": {"value": job_rate(1, world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": bytes_io,
                    "d2h_bytes_per_step": bytes_io},
            "gpu_launches": info_mixed.launches * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    for p in plans.values():
        p.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
