#!/usr/bin/env python3
"""Time-to-solution benchmark of the GB300 pipelined BiCGStab library.

Workload: 3-D convection-diffusion, 7-point first-order upwind stencil on a
256^3 grid (16,777,216 unknowns), velocity (20 sin y, 20 cos z, 20 sin x),
Dirichlet boundary, FP64; x* ~ U[-1, 1] (SplitMix64, seed 0), b = A x*,
x0 = 0. One step = one complete pipelined BiCGStab solve (Algorithm 9 with
residual replacement every 50 iterations) to ||r||/||r0|| <= 1e-8, stencil
form, inputs resident in HBM. The same line reports standard BiCGStab
(Algorithm 7) and the CSR form of the same matrix for comparison, the
end-to-end time through the host-buffer C entry point, the roofline of the
solver kernel and the CPU oracle timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-rel.res 1e-8 and HBM GB/s per iter, p-BiCGStab vs BiCGStab, 1 GB300"
RTOL = 1e-8
REPLACE_PERIOD = 50
MAXIT = 20000
SEED = 0
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak derived from unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM
# x 2 flop x 2.07 GHz (the 2 FMA/clk/SM is NVIDIA's 1.25 TFLOP/s GB300 FP64
# figure divided by 152 SMs and 2.07 GHz; a DFMA throughput loop measured
# 1.19 TFLOP/s on a GB300).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Oracle iteration counts on this workload (python -m oracle.full_solve_iterations),
# used to scale the CPU baseline's per-iteration time to a whole solve.
ORACLE_ITERS = {"pbicgstab_rr50": 415, "bicgstab": 352}
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the solver kernel on this workload, from a one-pass ncu capture of the full
# launch, valid only for the kernel sources it was taken on: SHA-256 over
# KERNEL_SOURCES.
KERNEL_SOURCES = ["paper_1612_01395_gb300/csrc/device_common.cuh", "paper_1612_01395_gb300/csrc/operators.cuh",
                  "paper_1612_01395_gb300/csrc/solvers.cuh"]
TRAFFIC_CAPTURE = {"bytes_per_launch": 984089911552 + 539640779776, "n": 16777216, "iters": 402, "grid": 1216,
                   "sources_sha256": "c891cf710bf10087f5daf028dee9bbdb2ad4ac66236c040ba9dc657ccf193849"}


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="grid points per axis")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-n", type=int, default=1024)
    ap.add_argument("--batch-systems", type=int, default=512)
    ap.add_argument("--mixed-n", type=int, default=192, help="grid points per axis of the mixed-precision case")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value):
    """Largest value over the ranks of the initialised process group (the
    timing rule of the replicas-only multi-GPU run); the value itself at N=1."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(n, form="stencil"):
    N = n ** 3
    return {"workload": f"3-D convection-diffusion {n}^3 (n={N}), 7-point upwind, velocity "
                        f"(20 sin y, 20 cos z, 20 sin x), {form} form, FP64, x*~U[-1,1] seed {SEED}, "
                        f"b=Ax*, x0=0, rtol {RTOL:g}, p-BiCGStab with residual replacement every "
                        f"{REPLACE_PERIOD} iterations",
            "n": N, "grid": [n, n, n], "form": form, "replace_period": REPLACE_PERIOD, "rtol": RTOL,
            "l2": "inputs larger than L2 (each vector 134 MB, working set > 1.6 GB); no flush"}


def nnz_of(n):
    return 7 * n ** 3 - 6 * n ** 2


def flops_per_launch(n, info):
    """Algorithmic FP64 flops of one solve: 2 flops per stored entry per SpMV
    plus, per iteration and unknown, 13 recurrence FMAs and 8 dot-product
    FMAs of Algorithm 9 (6 from the paper + ||r|| and ||q||), at 2 flops each."""
    N = n ** 3
    return info["spmvs"] * 2.0 * nnz_of(n) + info["iters"] * 2.0 * (13 + 8) * N


def batched_flops(sizes, nnz, iters, n_repl):
    """Algorithmic FP64 flops of one batched launch. Per system: 2 flops per
    stored entry per SpMV (r_0 = b - A x_0 and w_0 = A r_0, two per iteration,
    three more per residual replacement, the true residual at the end) plus
    42 flops per row and iteration (the recurrences and dot products of
    Algorithm 9, as in flops_per_launch)."""
    import numpy as np
    sizes, nnz = np.asarray(sizes, dtype=np.float64), np.asarray(nnz, dtype=np.float64)
    iters, n_repl = np.asarray(iters, dtype=np.float64), np.asarray(n_repl, dtype=np.float64)
    spmvs = 3.0 + 2.0 * iters + 3.0 * n_repl
    return float(np.sum(spmvs * 2.0 * nnz + iters * 2.0 * (13 + 8) * sizes))


def bytes_per_iter(n, form="stencil"):
    """Algorithmic HBM bytes per iteration of Algorithm 9: 23 N-vector passes
    (phase A reads w r p s z v r0, writes t p s z; phase B reads z x p r s w t
    r0, writes v x r w), each vector once; plus the matrix per SpMV for CSR
    (12 bytes per entry + 4 per row pointer)."""
    N = n ** 3
    b = 23 * 8 * N
    if form == "csr":
        b += 2 * (12 * nnz_of(n) + 4 * (N + 1))
    return b


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_inputs(n, need_csr):
    from paper_1612_01395_gb300 import problems as P
    st = P.cd3d_trig(n)
    A = P.stencil_to_csr(st) if need_csr else None
    xs = P.splitmix64_uniform(SEED, n ** 3)
    return st, A, xs


# ------------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------------

def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_sample(A, b, method, iters_lo=2, iters_hi=52, omp=False):
    """Seconds per oracle iteration and fixed overhead, from two fixed-iteration
    runs (iters_lo and iters_hi iterations); omp=True times the OpenMP build."""
    import oracle
    fn = oracle.pbicgstab if method == "pbicgstab" else oracle.bicgstab
    kw = {"replace_period": REPLACE_PERIOD} if method == "pbicgstab" else {}
    t = []
    for k in (iters_lo, iters_hi):
        t0 = time.perf_counter()
        fn(A, b, rtol=0.0, maxit=k, fixed_iters=k, omp=omp, **kw)
        t.append(time.perf_counter() - t0)
    per_iter = (t[1] - t[0]) / (iters_hi - iters_lo)
    overhead = max(t[0] - iters_lo * per_iter, 0.0)
    return per_iter, overhead, t[0] + t[1]


def cpu_baseline(A, b, gpu_iters):
    """The FP64 C oracle on the host cores: one complete solve (Algorithm 9,
    replacement every 50, to rtol 1e-8) with the OpenMP build on all cores,
    measured; and the single-threaded parity build on 2- and 52-iteration
    runs, its per-iteration time scaled to the oracle's iteration count
    (labelled extrapolated)."""
    import oracle
    model = cpu_model()
    threads = oracle.num_threads(omp=True)
    t0 = time.perf_counter()
    full = oracle.pbicgstab(A, b, rtol=RTOL, maxit=MAXIT, replace_period=REPLACE_PERIOD, omp=True)
    t_full = time.perf_counter() - t0
    per_iter, overhead, spent = oracle_sample(A, b, "pbicgstab")
    iters = ORACLE_ITERS["pbicgstab_rr50"] or gpu_iters
    return {"value": t_full, "unit": "s", "cores": threads, "kind": "oracle", "cpu_model": model,
            "sample": f"one complete solve of the full {A.n}-unknown system (CSR assembly of the same stencil) by "
                      f"the OpenMP build of the FP64 C oracle on {threads} threads: {full.iters} iterations to a "
                      f"true rel.res of {full.rel_res_true:.2e}, measured (not extrapolated)",
            "iters": full.iters, "status": int(full.status),
            "single_thread": {"value": overhead + iters * per_iter, "unit": "s", "cores": 1,
                              "s_per_iter": per_iter, "extrapolated": True,
                              "sample": f"2 and 52 fixed iterations of the single-threaded parity build "
                                        f"({spent:.1f} s of CPU work), per-iteration time scaled to {iters} "
                                        f"iterations (the oracle's own count)"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    n = args.n
    import oracle
    st, A, xs = build_inputs(n, need_csr=True)
    b = oracle.spmv(A, xs)
    threads = oracle.num_threads(omp=True)
    vals = []
    for s in range(args.warmup + args.steps):
        per_iter, overhead, spent = oracle_sample(A, b, "pbicgstab", 2, 52, omp=True)
        iters = ORACLE_ITERS["pbicgstab_rr50"] or 0
        v = overhead + iters * per_iter if iters else per_iter
        if s >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    unit = "s" if ORACLE_ITERS["pbicgstab_rr50"] else "s/iter"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(n), parallelism="replicas only" if world > 1 else "single GPU"),
            "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
                             "cpu_model": cpu_model(), "extrapolated": True,
                             "sample": "per step: 2 and 52 fixed iterations of the OpenMP build of the FP64 C "
                                       f"oracle (Algorithm 9) on {threads} threads on the full system, applied "
                                       "through the CSR assembly of the same stencil (identical values); "
                                       "per-iteration time scaled to the oracle's own iteration count"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------

def timed_solves(solver, bd, x, steps, method, rr, barrier):
    """Run `steps` solves bracketed by barrier + synchronize; returns (elapsed s, infos)."""
    import torch
    from paper_1612_01395_gb300 import native
    stream = torch.cuda.current_stream()
    infos = []
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        x.zero_()
        if method == "pipelined":
            st, info = native.pbicgstab_solve(solver.h, bd.data_ptr(), x.data_ptr(), RTOL, MAXIT, rr)
        else:
            st, info = native.bicgstab_solve(solver.h, bd.data_ptr(), x.data_ptr(), RTOL, MAXIT)
        if st != native.PBCG_OK:
            raise RuntimeError(f"solve failed: {native.STATUS_NAMES.get(st)} {native.pbicgstab_last_error()}")
        infos.append(info.as_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / 1e3, infos


def small_2d_case(barrier, m=64, steps=20):
    """The latency-bound workload: 2-D convection-diffusion on an m x m grid,
    velocity (10, 10), CSR form, x* ~ U[-1,1], b = A x*, x0 = 0, both methods
    to rtol 1e-8 (no replacement); mean time of `steps` solves after a warm-up."""
    import torch
    from paper_1612_01395_gb300 import native, problems as P
    A = P.stencil_to_csr(P.cd2d_constant(m, (10.0, 10.0)))
    s = native.Solver.from_csr(A)
    b = s.spmv(torch.from_numpy(P.splitmix64_uniform(SEED, A.n)).cuda())
    x = torch.zeros_like(b)
    out = {"workload": f"2-D convection-diffusion {m}^2 (n={A.n}), velocity (10,10), CSR (nnz={A.nnz}), rtol {RTOL:g}"}
    for method in ("pipelined", "standard"):
        timed_solves(s, b, x, 3, method, 0, barrier)
        el, inf = timed_solves(s, b, x, steps, method, 0, barrier)
        r = summarize(el, inf, steps)
        out["pbicgstab" if method == "pipelined" else "bicgstab"] = {
            k: r[k] for k in ("value", "iters", "ms_per_iter", "rel_res_true", "grid", "grid_syncs")}
    out["speedup_p_vs_bicgstab"] = out["bicgstab"]["value"] / out["pbicgstab"]["value"]
    s.close()
    return out


def size_sweep(sizes=(16, 32, 48, 64, 96, 128, 192, 256), iters=100):
    """Time per iteration of p-BiCGStab and BiCGStab on the n^3 convection-
    diffusion stencil, 100 fixed iterations each (the same work for both
    methods whatever their convergence): where the method pays on one GPU.
    Small n is bound by the grid-wide synchronisations (2 per iteration
    against 3 or 5), large n by FP64 arithmetic (Algorithm 9 does 1.3x the
    FP64 work of Algorithm 7 per iteration)."""
    import torch
    from paper_1612_01395_gb300 import native, problems as P
    out = {}
    for n in sizes:
        st = P.cd3d_trig(n)
        s = native.Solver.from_stencil(st)
        b = s.spmv(torch.from_numpy(P.splitmix64_uniform(SEED, st.n)).cuda())
        row = {}
        for method in ("pipelined", "standard"):
            kw = dict(rtol=0.0, maxit=iters, fixed_iters=iters, method=method)
            s.solve(b, **kw)
            infos = [s.solve(b, **kw)[1] for _ in range(3)]
            us = statistics.median(1e3 * i["kernel_ms"] / max(i["iters"], 1) for i in infos)
            row["pbicgstab_us_per_iter" if method == "pipelined" else "bicgstab_us_per_iter"] = us
        row["p_over_plain_time_per_iter"] = row["pbicgstab_us_per_iter"] / row["bicgstab_us_per_iter"]
        out[str(st.n)] = row
        s.close()
    return out


def jacobi_case(st, bd, x, barrier):
    """Right Jacobi preconditioning (Algorithms 11 and 10, M = diag(A)) on the
    same system and tolerance, one timed solve each after a warm-up."""
    from paper_1612_01395_gb300 import native
    s = native.Solver.from_stencil(st, prec=native.PBCG_PREC_JACOBI)
    out = {}
    for method, rr in (("pipelined", REPLACE_PERIOD), ("standard", 0)):
        timed_solves(s, bd, x, 1, method, rr, barrier)
        el, inf = timed_solves(s, bd, x, 1, method, rr, barrier)
        r = summarize(el, inf, 1)
        out["pbicgstab_jacobi" if method == "pipelined" else "bicgstab_jacobi"] = {
            k: r[k] for k in ("value", "iters", "ms_per_iter", "rel_res_true", "grid")}
    s.close()
    return out


def grid_sensitivity(solver, bd, x, grid):
    """Both methods to rtol at 4 to 9 blocks per SM (each method up to its
    own co-resident maximum). The grid fixes the order in which dot products
    are summed, and BiCGStab's trajectory depends on rounding: the counts to
    1e-8 move by 10-20 %. So the two methods are also compared by the median
    of their time to rtol over the grids on which both ran (a secondary
    figure; the headline compares each method at its own default launch)."""
    import torch
    from paper_1612_01395_gb300 import native
    per_sm = torch.cuda.get_device_properties(0).multi_processor_count
    out = {}
    for g in [k * per_sm for k in range(4, 10)]:
        row = {}
        for method in ("pipelined", "standard"):
            x.zero_()
            if method == "pipelined":
                st, info = native.pbicgstab_solve(solver.h, bd.data_ptr(), x.data_ptr(), RTOL, MAXIT, REPLACE_PERIOD,
                                                  grid=g)
            else:
                st, info = native.bicgstab_solve(solver.h, bd.data_ptr(), x.data_ptr(), RTOL, MAXIT, grid=g)
            if info.grid != g:   # above this method's co-resident maximum
                continue
            row[method] = {"iters": info.iters, "ms": info.kernel_ms, "ms_per_iter": info.kernel_ms / max(info.iters, 1),
                           "status": native.STATUS_NAMES.get(st)}
        out[str(g)] = row
    # medians over the grids on which both methods ran and converged (the same summation-order set)
    common = [g for g, row in out.items() if "pipelined" in row and "standard" in row
              and row["pipelined"]["status"] == "OK" and row["standard"]["status"] == "OK"]
    med = {m: statistics.median(out[g][m]["ms"] for g in common) / 1e3 if common else None
           for m in ("pipelined", "standard")}
    out["common_grids"] = [int(g) for g in common]
    out["median_s_over_common_grids"] = med
    out["median_p_over_plain"] = (med["pipelined"] / med["standard"]
                                  if med["pipelined"] and med["standard"] else None)
    return out


def summarize(elapsed, infos, steps):
    its = [i["iters"] for i in infos]
    sec = elapsed / steps
    return {"value": sec, "iters": int(statistics.median(its)), "ms_per_iter": 1e3 * sec / statistics.median(its),
            "rel_res_true": max(i["rel_res_true"] for i in infos),
            "kernel_ms": statistics.mean(i["kernel_ms"] for i in infos),
            "grid_syncs": infos[0]["grid_syncs"], "spmvs": infos[0]["spmvs"], "grid": infos[0]["grid"]}


def mixed_precision_case(n, steps, barrier):
    """FP64 refinement around FP32 (and BF16-valued) Algorithm 9 against all-FP64
    p-BiCGStab, both to a true relative residual of 1e-10, on the n^3
    convection-diffusion system in CSR form and in stencil form.

    Inner solves stop at their tolerance or after a cap of iterations (a
    restart): an FP32 Krylov solve can stagnate far above its tolerance, and
    the next step's FP64 residual restarts it. The FP32 inner iteration counts
    move by 15-25 % with the summation order (the grid), so each setting is
    also solved at two more grid sizes and the median reported beside the
    default-grid time."""
    import statistics as stats
    import torch
    from paper_1612_01395_gb300 import native, problems as P
    st = P.cd3d_trig(n)
    A = P.stencil_to_csr(st)
    N = A.n
    solvers = {"csr": native.Solver.from_csr(A), "stencil": native.Solver.from_stencil(st)}
    bd = solvers["stencil"].spmv(torch.from_numpy(P.splitmix64_uniform(SEED, N)).cuda())
    vals = {"fp32": torch.as_tensor(A.val).cuda().to(torch.float32),
            "bf16": torch.as_tensor(A.val).cuda().to(torch.bfloat16)}
    out = {"workload": f"3-D convection-diffusion {n}^3 (n={N}), CSR (nnz={A.nnz}) and stencil forms, "
                       f"true rel.res 1e-10"}

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            res = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / k, res

    k = max(1, min(steps, 3))
    x64 = {}
    for form, s in solvers.items():
        sec, (x, info) = timed(lambda: s.solve(bd, rtol=1e-10, maxit=MAXIT, replace_period=REPLACE_PERIOD), k)
        x64[form] = x
        out[f"{form}_fp64_pbicgstab"] = {"value": sec, "iters": info["iters"], "rel_res_true": info["rel_res_true"],
                                         "status": native.STATUS_NAMES[info["status"]]}
    cases = [("csr", "fp32", 1e-1, 50), ("csr", "fp32", 3e-2, 150), ("stencil", "fp32", 1e-1, 50),
             ("stencil", "fp32", 3e-2, 150), ("csr", "bf16", 1e-2, 150)]
    for form, vt, tau, cap in cases:
        s = solvers[form]
        v = None if form == "stencil" else vals[vt]
        typ = native.PBCG_VALUES_BF16 if vt == "bf16" else native.PBCG_VALUES_F32
        name = f"{form}_mixed_{vt}_inner{tau:g}_cap{cap}"

        def run(grid=0):
            return s.solve_mixed(bd, v, typ, rtol=1e-10, max_outer=60, inner_rtol=tau, inner_maxit=cap, grid=grid)
        try:
            sec, (xm, im) = timed(run, k)
        except native.PbcgError as e:
            out[name] = {"error": str(e)}
            continue
        ref = out[f"{form}_fp64_pbicgstab"]["value"]
        per_grid = {"default": sec}
        if im["status"] == native.PBCG_OK:
            for g in (1292, 1216, 1140, 1064):   # 8.5 to 7 blocks per SM, below the default 9: other summation orders
                _, ig = run(g)
                per_grid[str(g)] = ig["kernel_ms"] / 1e3
        median = stats.median(per_grid.values())
        err = float(torch.linalg.norm(xm - x64[form]) / torch.linalg.norm(x64[form]))
        mat_bytes = 0 if form == "stencil" else 2 * ((4 if vt == "fp32" else 2) + 4) * A.nnz + 8 * (N + 1)
        inner_bytes = 24 * 4 * N + mat_bytes   # FP32 vectors (+ low-precision CSR), per inner iteration
        out[name] = {"value": sec, "outer": im["outer"], "inner_iters": im["inner_iters"], "inner_maxit": cap,
                     "rel_res_true": im["rel_res_true"], "status": native.STATUS_NAMES[im["status"]],
                     "returned_best_earlier_iterate": bool(im["restored"]),
                     "rel_error_vs_fp64": err, "speedup_vs_fp64": ref / sec,
                     "ms_per_inner_iter": im["kernel_ms"] / max(1, im["inner_iters"]),
                     "s_per_grid": per_grid, "median_s_over_grids": median, "median_speedup_vs_fp64": ref / median,
                     "inner_gbs_est": inner_bytes * im["inner_iters"] / (im["kernel_ms"] / 1e3) / 1e9}
    for s in solvers.values():
        s.close()
    return out


def batched_case(nsys, steps, barrier):
    """512 random unsymmetric systems (sizes log-uniform in 1k-64k, 8-32
    off-diagonals per row, diagonal 1.1 x row sum) solved to rtol 1e-8 each in
    one launch, captured in a CUDA graph and replayed; compared with solving
    the same systems one after another with the single-system solver."""
    import torch
    import numpy as np
    from paper_1612_01395_gb300 import native, problems as P
    t0 = time.perf_counter()
    B = P.random_batch(nsys=nsys, seed=SEED)
    gen_s = time.perf_counter() - t0
    bs = native.BatchSolver(B)
    b = torch.from_numpy(B.b).cuda()
    x = torch.zeros_like(b)
    # the library's autotuner picks the launch shape (cluster size, threshold)
    cs, cm, tune_ms = bs.autotune(b, x, rtol=RTOL, maxit=MAXIT)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        x.zero_()
        bs.launch(b, x, rtol=RTOL, maxit=MAXIT, stream=s, cluster_size=cs, cluster_min_rows=cm)
    g.replay()
    torch.cuda.synchronize()
    k = max(1, min(steps, 3))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(k):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / k
    res = bs.fetch_results()
    # the same systems one at a time through the single-system entry point (first 64 systems, scaled)
    m = min(64, B.nsys)
    t_single, its_single = 0.0, 0
    for sidx in range(m):
        A = B.system(sidx)
        r0, r1 = int(B.row_offset[sidx]), int(B.row_offset[sidx + 1])
        sv = native.Solver.from_csr(A)
        bb = b[r0:r1].contiguous()
        sv.solve(bb, rtol=RTOL, maxit=MAXIT)
        _, inf = sv.solve(bb, rtol=RTOL, maxit=MAXIT)
        t_single += inf["kernel_ms"] / 1e3
        its_single += inf["iters"]
        sv.close()
    frac = float(B.sizes[:m].sum()) / float(B.sizes.sum())
    nnz_sys = B.rowptr[B.row_offset[1:]].astype(np.int64) - B.rowptr[B.row_offset[:-1]].astype(np.int64)
    fl = batched_flops(B.sizes, nnz_sys, res["iters"], res["n_replacements"])
    achieved_tf = fl / sec / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tf / FP64_PEAK_TFLOPS, "kernel": "batched_kernel", "flops_per_launch": fl,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz"}
    return {"workload": f"{B.nsys} random sparse systems, sizes log-uniform 1k-64k (total {B.total_rows} rows, "
                        f"{int(B.rowptr[-1])} nnz), rtol {RTOL:g}, one launch replayed from a CUDA graph",
            "value": sec, "unit": "s", "systems_converged": int(np.sum(res["status"] == native.PBCG_OK)),
            "launch_shape": {"cluster_size": cs, "cluster_min_rows": cm, "autotuner_ms": tune_ms},
            "iters_total": int(res["iters"].sum()), "iters_max": int(res["iters"].max()),
            "max_rel_res_true": float(res["rel_res_true"].max()), "generation_s": gen_s,
            "single_system_solver_est_s": t_single / frac if frac > 0 else None,
            "single_system_sample": f"first {m} systems (largest) solved one per launch, {frac:.2%} of the rows, "
                                    f"scaled by rows",
            "speedup_vs_single_system_solver": (t_single / frac) / sec if frac > 0 else None,
            "roofline": roofline}


def adjoint_case(n, barrier):
    """Reverse-mode gradient of L = 0.5 ||x - x_target||^2, x = A^{-1} b, on the
    n^2 convection-diffusion system with per-cell velocity c ~ U[0, 50]:
    forward solve + adjoint solve with A^T (pipelined BiCGStab, rtol 1e-13,
    replacement every 50), checked against central finite differences two ways:

    * the configured check: step h = 1e-6 on 32 random coordinates (16 of b,
      16 of the matrix values); each perturbed solution is the unperturbed x*
      plus a correction solved to rtol 1e-10 of its own right-hand side, so
      the correction's error scales with h and the difference quotient keeps
      its accuracy; per-coordinate relative errors |fd - g| / |g|, no floor;
    * large steps from cold starts: dL/db with h = 1e-2 (L is quadratic in b),
      dL/dvalues by one Richardson step over 5e-3 and 1e-2, errors against
      |g| + 1e-3 max|g|, on 16 coordinates."""
    import torch
    import numpy as np
    from paper_1612_01395_gb300 import native, problems as P
    from paper_1612_01395_gb300.adjoint import CSRStructure, sparse_solve
    A = P.stencil_to_csr(P.cd2d_field(n, seed=SEED))
    st = CSRStructure(A.rowptr, A.col)
    vals0 = torch.from_numpy(A.val).cuda()
    b0 = torch.from_numpy(P.splitmix64_uniform(SEED + 2, A.n)).cuda()
    xt = torch.from_numpy(P.splitmix64_uniform(SEED + 3, A.n)).cuda()

    def loss(vals, bb):
        x = sparse_solve(vals, bb, st, rtol=1e-13)
        return 0.5 * ((x - xt) ** 2).sum()

    vals = vals0.clone().requires_grad_(True)
    bb = b0.clone().requires_grad_(True)
    loss(vals, bb).backward()                        # warm-up
    torch.cuda.synchronize()
    barrier()
    vals = vals0.clone().requires_grad_(True)
    bb = b0.clone().requires_grad_(True)
    t0 = time.perf_counter()
    L = loss(vals, bb)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    L.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    gb, gv = bb.grad.cpu().numpy(), vals.grad.cpu().numpy()

    # configured check: h = 1e-6. Each perturbed solution is x* + d with
    # A' d = b' - A' x* (A', b' the perturbed system), solved from d = 0 to rtol
    # 1e-10 of its own right-hand side; the numerator of the central difference,
    # L(+) - L(-), is evaluated without cancellation for this quadratic loss:
    # (x* - x_t).(d+ - d-) + (|d+|^2 - |d-|^2) / 2.
    with torch.no_grad():
        xstar = sparse_solve(vals0, b0, st, rtol=1e-13)
    nws = native.pbicgstab_workspace_bytes(A.n)
    ws = torch.empty(nws // 8 + 64, dtype=torch.float64, device="cuda")
    wsp = (ws.data_ptr() + 255) // 256 * 256
    stream = torch.cuda.current_stream().cuda_stream

    def correction(v, bvec):
        h = native.pbicgstab_create_csr(A.n, A.nnz, st.rowptr.data_ptr(), st.col.data_ptr(), v.data_ptr(),
                                        native.PBCG_PREC_NONE, wsp, nws, stream)
        ax = torch.empty_like(xstar)
        native.pbicgstab_spmv(h, xstar.data_ptr(), ax.data_ptr())
        rhs = bvec - ax
        d = torch.zeros_like(xstar)
        rc, info = native.pbicgstab_solve(h, rhs.data_ptr(), d.data_ptr(), 1e-10, MAXIT, REPLACE_PERIOD)
        native.pbicgstab_destroy(h)
        if rc != native.PBCG_OK:
            raise RuntimeError(f"correction solve failed: {native.STATUS_NAMES.get(rc)}")
        return d

    def central_numerator(vp, bp, vm, bm):
        dp, dm = correction(vp, bp), correction(vm, bm)
        return float(torch.dot(xstar - xt, dp - dm) + 0.5 * (torch.dot(dp, dp) - torch.dot(dm, dm)))

    hcfg = 1e-6
    rel_cfg = []
    t3 = time.perf_counter()
    with torch.no_grad():
        for i in (P.splitmix64(SEED + 21, 16) % np.uint64(A.n)).astype(int):
            e = torch.zeros_like(b0)
            e[i] = hcfg
            fd = central_numerator(vals0, b0 + e, vals0, b0 - e) / (2 * hcfg)
            rel_cfg.append(("b", int(i), float(gb[i]), fd, abs(fd - gb[i]) / abs(gb[i])))
        for k in (P.splitmix64(SEED + 22, 16) % np.uint64(A.nnz)).astype(int):
            e = torch.zeros_like(vals0)
            e[k] = hcfg
            fd = central_numerator(vals0 + e, b0, vals0 - e, b0) / (2 * hcfg)
            rel_cfg.append(("val", int(k), float(gv[k]), fd, abs(fd - gv[k]) / abs(gv[k])))
    t4 = time.perf_counter()
    rels = [r[4] for r in rel_cfg]

    # large-step check from cold starts
    worst = 0.0
    sb, sv = 1e-3 * np.abs(gb).max(), 1e-3 * np.abs(gv).max()

    def central(vals, bb, e, h):
        return (float(loss(vals + e[0], bb + e[1])) - float(loss(vals - e[0], bb - e[1]))) / (2 * h)

    zv, zb = torch.zeros_like(vals0), torch.zeros_like(b0)
    with torch.no_grad():
        for i in (P.splitmix64(SEED + 11, 8) % np.uint64(A.n)).astype(int):
            e = torch.zeros_like(b0)
            e[i] = 1e-2
            fd = central(vals0, b0, (zv, e), 1e-2)
            worst = max(worst, abs(fd - gb[i]) / (abs(gb[i]) + sb))
        for k in (P.splitmix64(SEED + 12, 8) % np.uint64(A.nnz)).astype(int):
            e1, e2 = torch.zeros_like(vals0), torch.zeros_like(vals0)
            e1[k], e2[k] = 5e-3, 1e-2
            fd = (4 * central(vals0, b0, (e1, zb), 5e-3) - central(vals0, b0, (e2, zb), 1e-2)) / 3
            worst = max(worst, abs(fd - gv[k]) / (abs(gv[k]) + sv))
    return {"workload": f"2-D convection-diffusion {n}^2 (n={A.n}), per-cell velocity (c, c), c ~ U[0,50]; "
                        f"L = 0.5||x - x_t||^2; gradients w.r.t. b and the {A.nnz} matrix values",
            "forward_s": t1 - t0, "backward_s": t2 - t1, "value": t2 - t0, "unit": "s",
            "fd_h1e-6": {"coordinates": len(rel_cfg), "max_rel_error": max(rels),
                         "median_rel_error": float(np.median(rels)),
                         "per_coordinate": [{"of": r[0], "index": r[1], "grad": r[2], "fd": r[3], "rel_error": r[4]}
                                            for r in rel_cfg],
                         "method": "central differences, h = 1e-6; each perturbed solution is x* + d with d "
                                   "solved to rtol 1e-10 of its own right-hand side b' - A' x*; L(+) - L(-) "
                                   "evaluated as (x* - x_t).(d+ - d-) + (|d+|^2 - |d-|^2)/2",
                         "s_per_coordinate": (t4 - t3) / len(rel_cfg)},
            "fd_large_steps": {"coordinates": 16, "max_rel_error": worst, "error_scale": "|g_k| + 1e-3 max|g|",
                               "method": "cold starts; b: h = 1e-2; values: Richardson over 5e-3 and 1e-2"}}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")

        def barrier():
            dist.barrier()
    else:
        torch.cuda.set_device(0)

        def barrier():
            pass

    from paper_1612_01395_gb300 import native
    native.build()
    n = args.n
    N = n ** 3
    want_cpu = (not args.no_cpu_baseline) and rank == 0 and world == 1
    st, A, xs = build_inputs(n, need_csr=(not args.no_compare) or want_cpu)

    solver = native.Solver.from_stencil(st)
    xd = torch.from_numpy(xs).cuda()
    bd = solver.spmv(xd)                       # b = A x* on the device
    x = torch.zeros_like(bd)

    # warm-up, then the timed region: K pipelined solves, stencil form
    timed_solves(solver, bd, x, args.warmup, "pipelined", REPLACE_PERIOD, barrier)
    clocks = ClockSampler(local)
    clocks.start()
    elapsed, infos = timed_solves(solver, bd, x, args.steps, "pipelined", REPLACE_PERIOD, barrier)
    clk = clocks.stop()
    elapsed = max_over_ranks(elapsed)
    main = summarize(elapsed, infos, args.steps)
    sec = main["value"]

    # roofline of the solver kernel (one cooperative launch per solve)
    kern_s = main["kernel_ms"] / 1e3
    fl = flops_per_launch(n, infos[0])
    achieved_tf = fl / kern_s / 1e12
    peaks = json.load(open(MEASURED_PEAKS)) if os.path.exists(MEASURED_PEAKS) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    bpi = bytes_per_iter(n)
    gbs = bpi * main["iters"] / kern_s / 1e9
    traffic = None
    if TRAFFIC_CAPTURE is not None and TRAFFIC_CAPTURE["sources_sha256"] == kernel_sources_sha256() \
            and TRAFFIC_CAPTURE["n"] == N and TRAFFIC_CAPTURE["iters"] == main["iters"] \
            and TRAFFIC_CAPTURE["grid"] == infos[0]["grid"]:
        traffic = TRAFFIC_CAPTURE["bytes_per_launch"]
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tf / FP64_PEAK_TFLOPS, "traffic": traffic,
                "kernel": "pbicgstab_kernel<StencilOp>",
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz",
                "flops_per_launch": fl,
                "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak,
                        "peak_source": hbm_src, "bytes_per_iter": bpi}}

    out = {"metric": METRIC, "value": sec, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(workload_config(n), parallelism="replicas only" if world > 1 else "single GPU"),
           "iters": main["iters"], "ms_per_iter": main["ms_per_iter"], "rel_res_true": main["rel_res_true"],
           "hbm_gbs_per_iter": gbs, "grid_syncs_per_solve": main["grid_syncs"], "grid": main["grid"],
           "roofline": roofline, "clocks": clk, "gpu_launches": args.steps,
           "create_s": {"stencil": solver.create_s}}

    # comparison: standard BiCGStab on the same form, and both methods on CSR
    if not args.no_compare:
        ksteps = max(1, min(args.steps, 3))
        _, _ = timed_solves(solver, bd, x, 1, "standard", 0, barrier)
        el, inf = timed_solves(solver, bd, x, ksteps, "standard", 0, barrier)
        plain = summarize(el, inf, ksteps)
        out["bicgstab"] = dict(plain, form="stencil")
        out["speedup_p_vs_bicgstab"] = plain["value"] / sec
        csolver = native.Solver.from_csr(A)
        out["create_s"]["csr"] = csolver.create_s   # includes the device-side structure check
        cmp_csr = {}
        for method, rr in (("pipelined", REPLACE_PERIOD), ("standard", 0)):
            timed_solves(csolver, bd, x, 1, method, rr, barrier)
            el, inf = timed_solves(csolver, bd, x, ksteps, method, rr, barrier)
            r = summarize(el, inf, ksteps)
            r["hbm_gbs_per_iter"] = bytes_per_iter(n, "csr") * r["iters"] / (r["kernel_ms"] / 1e3) / 1e9 \
                if method == "pipelined" else None
            if r["hbm_gbs_per_iter"] is not None:
                r["hbm_frac_of_measured_peak"] = r["hbm_gbs_per_iter"] / hbm_peak
            cmp_csr["pbicgstab" if method == "pipelined" else "bicgstab"] = r
        out["csr"] = cmp_csr
        csolver.close()
        out["grid_sensitivity"] = grid_sensitivity(solver, bd, x, main["grid"])
        out["jacobi"] = jacobi_case(st, bd, x, barrier)
        out["size_sweep"] = size_sweep()
        slower = [int(k) for k, v in out["size_sweep"].items() if v["p_over_plain_time_per_iter"] > 1.0]
        out["size_sweep_crossover_n"] = min(slower) if slower else None   # smallest n where p-BiCGStab is slower per iteration
        out["small_2d"] = small_2d_case(barrier)

    if not args.no_mixed:
        out["mixed_precision"] = mixed_precision_case(args.mixed_n, args.steps, barrier)
    if not args.no_batched:
        out["batched"] = batched_case(args.batch_systems, args.steps, barrier)
    if not args.no_adjoint:
        out["adjoint"] = adjoint_case(args.adjoint_n, barrier)

    # end to end through the host-buffer C entry point: H2D b and x0, solve, D2H x
    hb = torch.from_numpy(bd.cpu().numpy()).pin_memory()
    hx = torch.zeros(N, dtype=torch.float64).pin_memory()
    e2e_times = []
    for s in range(1 + args.steps):
        hx.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stt, _ = native.pbicgstab_solve_host(solver.h, 0, hb.data_ptr(), hx.data_ptr(), RTOL, MAXIT, REPLACE_PERIOD)
        t1 = time.perf_counter()
        if stt != native.PBCG_OK:
            raise RuntimeError("host solve failed")
        if s > 0:
            e2e_times.append(t1 - t0)
    out["e2e"] = {"value": statistics.median(e2e_times), "unit": "s", "h2d_bytes_per_step": 2 * 8 * N,
                  "d2h_bytes_per_step": 8 * N + ctypes.sizeof(native.PbcgInfo)}

    if want_cpu:
        import oracle
        b_host = oracle.spmv(A, xs)
        out["cpu_baseline"] = cpu_baseline(A, b_host, main["iters"])
    else:
        out["cpu_baseline"] = None
    solver.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
