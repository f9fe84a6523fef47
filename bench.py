"""Benchmark: time to solve the 128^3 lognormal-diffusivity Poisson system
(random + RCM ordering) to relative residual 1e-8 on one GB300.

A step is one complete solve through the C ABI (repacked matrix resident in
HBM, right-hand side resident): the mixed-precision pipelined PCG (float
recurrences, FP64 solution and residual replacement) is the headline; plain
FP64 Jacobi-PCG and FP64 pipelined PCG are timed the same way beside it.
Every step starts with an L2 flush (a 256 MB write, outside the timed
events); each step is timed with CUDA events on the solve's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--size S] [--skip-fp64]

--impl reference times the oracle's FP64 Jacobi-PCG (the same C source built
with OpenMP, every host core) solving the same system to 1e-8, one complete
solve per step.  Our arm also reports the plain single-threaded oracle's
complete solve (cpu_baseline), the error of every result against the
oracle's tight FP64 solution (computed after the timed legs), and the FP64
rate of cuBLAS DGEMM on this GPU (the FP64 solvers' arithmetic bound).
Under torchrun (N > 1) every rank solves its own replica (no data exchange:
the single-system solve is not partitioned here) and rank 0 prints the
maximum over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "128³ Poisson solve to 1e-8 rel. res.: s and HBM GB/s, mixed vs FP64 PCG"
TOL = 1e-8


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---- ncu traffic of the dominant kernel ----------------------------------------
PROFILE = os.path.join(ROOT, "profiles", "k_mixed_poisson128.md")


def source_digest():
    """sha256 over the sources that build the single-system solve kernels and
    their matrix layout (the repack): a profile's DRAM counters describe the
    kernel only while this digest is unchanged."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1505_07630_gb300", "csrc")
    for name in ("ldupcg_impl.cuh", "setup.cu", "setup_kernels.cuh", "solve.cu",
                 "solve_kernels.cuh"):
        h.update(name.encode())
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(slice_rows=None):
    """(dram bytes per launch, iterations) from the committed ncu summary, or
    None when the kernel sources changed since that capture or it was taken
    with another slice height."""
    try:
        fields = {}
        with open(PROFILE) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
        if fields.get("source_sha256") != source_digest():
            return None
        if slice_rows is not None and int(fields.get("slice_rows", -1)) != slice_rows:
            return None
        return float(fields["dram_bytes_per_launch"]), int(fields["iterations"])
    except (OSError, KeyError, ValueError):
        return None


# ---- algorithmic bytes (one launch = one solve) ------------------------------
# Per cell, with f = 2F/n off-diagonal entries per row (actual, padding
# excluded), float values/indices 4 B, double 8 B; vectors counted once per
# pass they are read or written, gathers once.
def bytes_mixed(n, F, iters, reps, col_bytes=4, deflated=False):
    """col_bytes: bytes per column index in the float loop (2 when the staged
    sweep reads 16-bit column offsets).  deflated: the constant-vector
    deflation's three float vectors in every sweep, and its FP64 coarse
    correction in every replacement."""
    f = 2.0 * F / n
    loop = f * (4 + col_bytes) + 6 * 4 + 6 * 4    # matrix (val32+col) + 6 reads + 6 writes
    rep = (24                                     # fold: xhat rw, xc rw
           + f * 12 + 8 + 8 + 8 + 8 + 4           # FP64 residual: val64+col, xhat, bhat, dg, r out
           + f * 8 + 4 + 4 + 4 + 4                # w = Ar, s = Ap
           + f * 8 + 4 + 4 + 8 + 8 + 4)           # z = As, rescale r, p, read w
    if deflated:
        loop += 3 * 4                             # w0, q0, t0 (float) read every sweep
        rep += 8 + 8 + 5 * 8 + 8 + 4 + 4          # w0 in, r out; xhat, r, w0, q0, dg in, xhat, r out; q0 in
    ends = 8 * 4 + 4 * 4 + 3 * 8                  # prep (b, x0 in; bhat, xhat out; zero 4 float) + unscale
    return n * (iters * loop + reps * rep + ends)


def bytes_mixed_preconditioned(n, F, iters, reps):
    """Algorithmic bytes of the FP32-inner pipelined PCG in its preconditioned
    form (the recurrences of Sec. 4.1 with M^-1 applied to separate vectors):
    per float iteration 4n (float diagonal) + 16F (2F float values and int32
    columns) + 80n (ten float vectors once each), per FP64 residual
    replacement 8n + 24F + 24n.  The library's scaled formulation needs no
    M^-1 vectors and 16-bit columns (bytes_mixed), so this count is larger
    than what the kernel has to move."""
    return iters * (4.0 * n + 16.0 * F + 80.0 * n) + reps * (8.0 * n + 24.0 * F + 24.0 * n)


# FP64 instructions per cell and iteration of k_pcg64 (the scaled product:
# about 6 FMAs for the off-diagonal slots and one add for the unit diagonal;
# (p, q), two updates, (r, r) and sum d r^2, the p update: 7 more)
PCG64_FP64_INSTR_PER_CELL = 13


def bytes_pcg64(n, F, iters, reps):
    f = 2.0 * F / n
    spmv = f * 12 + 8 + 8                         # q = A p: val64+col, p, q out
    upd = 5 * 8 + 2 * 8                           # x, p, r, q, dg in; x, r out
    pup = 3 * 8                                   # p = r + beta p
    res = f * 12 + 8 + 8 + 8 + 8                  # true residual
    return n * (iters * (spmv + upd + pup) + reps * res + 6 * 8)


def bytes_pipe64(n, F, iters, reps):
    f = 2.0 * F / n
    loop = f * 12 + 7 * 8 + 6 * 8                 # matrix + w,z,s,p,x,r,dg in; 6 out
    rep = (f * 12 + 4 * 8 + 8) + (f * 12 + 2 * 8 + 2 * 8) + (f * 12 + 4 * 8 + 8)
    return n * (iters * loop + reps * rep + 8 * 8)


# ---- clocks ----------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ldupcg_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---- ranks (one process per GPU; replicas: no collective on the data path) --
class Ranks:
    """Rank layout of a torchrun launch, or of a single process."""

    def __init__(self, env=None):
        env = os.environ if env is None else env
        self.world = int(env.get("WORLD_SIZE", "1"))
        self.rank = int(env.get("RANK", "0"))
        self.local = int(env.get("LOCAL_RANK", "0"))


def init_ranks(backend):
    """(ranks, process group module or None): the group is set up only for
    more than one rank, from the MASTER_* variables torchrun exports."""
    r = Ranks()
    dist = None
    if r.world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return r, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def job_seconds(local_seconds, dist, device="cpu"):
    """The job's time: the largest of every rank's own timed total."""
    if dist is None:
        return local_seconds
    import torch
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def emit(line, ranks):
    """Rank 0 prints the one JSON line of the run."""
    if ranks.rank == 0:
        print(json.dumps(line), flush=True)


# ---- the oracle arm --------------------------------------------------------
def oracle_solve(sys_, omp):
    """(seconds, result) of one complete FP64 Jacobi-PCG solve to TOL by the
    oracle: the plain single-threaded build, or (omp) the OpenMP build on
    every host core."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.pcg(sys_, tol=TOL, omp=omp)
    return time.perf_counter() - t0, r


# the workload both arms solve: the 128^3 lognormal Poisson system to relative residual 1e-8
WORKLOAD = ("poisson {size}^3 lognormal(0,1) k, harmonic faces, random+RCM order, Dirichlet "
            "x-walls; Jacobi-preconditioned CG to 1e-8")


def run_reference(args):
    ranks = Ranks()
    if ranks.rank != 0:
        return   # the oracle arm runs on rank 0 alone; other ranks exit without work
    import ldu_cases as lc
    import oracle
    s = lc.config2(s=args.size, seed=0)
    oracle.lib(omp=True)
    cores = oracle.threads(omp=True)
    for _ in range(args.warmup):
        oracle_solve(s, omp=True)
    per, res = [], None
    for _ in range(args.steps):
        t, res = oracle_solve(s, omp=True)
        per.append(t)
    value = statistics.mean(per)
    sample = (f"one complete FP64 Jacobi-PCG solve of the {args.size}^3 case to 1e-8 per step "
              f"({res.iters} iterations), the oracle's C source built with OpenMP on {cores} "
              f"host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(size=args.size), "cells": s.n, "faces": s.nfaces,
                   "solver": "FP64 Jacobi-PCG, the oracle (C, OpenMP over the host cores)"},
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_iters": res.iters, "oracle_relres": res.relres,
        "step_s_min_median_max": [min(per), statistics.median(per), max(per)],
    }
    emit(line, ranks)


def fp64_dgemm_tflops(dev, n=4096, reps=5):
    """FP64 rate of this GPU as cuBLAS reaches it: torch.matmul of two n x n
    float64 matrices, 2 n^3 flops, best of reps, CUDA events."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    torch.cuda.synchronize(dev)
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return 2.0 * n ** 3 / best / 1e12


def rel_err(x, xs):
    import numpy as np
    return float(np.linalg.norm(np.asarray(x) - xs) / np.linalg.norm(xs))


def accuracy_report(s, solutions, batched_x=None, piso=None):
    """The error of every result against the oracle's tight FP64 solution
    x* (Jacobi-PCG of the OpenMP build to the limit of FP64), computed after
    the timed legs.  solutions: name -> x of the 128^3 system; batched_x:
    (systems, concatenated x); piso: (system, b, p)."""
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    xs, rr, kappa = oracle.reference_solution(s)
    out = {"reference": {"relres": rr, "kappa_est": kappa,
                         "solver": "oracle FP64 Jacobi-PCG (OpenMP build) to 4e-15 or stagnation"},
           "errors": {k: rel_err(x, xs) for k, x in solutions.items()}}
    if batched_x is not None:
        systems, xb = batched_x
        off, errs = 0, []
        for q in systems:
            xq, _, _ = oracle.reference_solution(q)
            errs.append(rel_err(xb[off:off + q.n], xq))
            off += q.n
        out["errors"]["batched_max"] = max(errs)
        out["errors"]["batched_median"] = float(np.median(errs))
    if piso is not None:
        sp, bp, pp = piso
        xq, rq, kq = oracle.reference_solution(sp, b=bp)
        out["errors"]["piso_pressure_last_step"] = rel_err(pp, xq)
        out["reference"]["piso_relres"] = rq
        out["reference"]["piso_kappa_est"] = kq
    out["seconds"] = time.perf_counter() - t0
    return out


# ---- our arm ---------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import ldu_cases as lc

    ranks, dist = init_ranks("nccl")
    world, rank, local = ranks.world, ranks.rank, ranks.local
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_07630_gb300 as pkg

    from paper_1505_07630_gb300 import autotune

    s = lc.config2(s=args.size, seed=0)
    n, F = s.n, s.nfaces
    # each solver at its own best layout (autotuned once, cached; untimed)
    cands = (args.slice_rows,) if args.slice_rows else (128, 64)
    fixed = {"rr_period": args.rr_period, "tau": args.tau} if args.rr_period else {}
    if args.slice_rows and args.rr_period:
        tune_m = dict(slice_rows=args.slice_rows, **fixed)   # fixed: no tuning
    else:
        tune_m = autotune.tune_single(s, "mixed", tol=TOL, slice_rows=cands, **fixed)
    # replacement rule: the tuned one, else the library's default (both 0)
    rr_m = args.rr_period or tune_m.get("rr_period", 0)
    tau_m = args.tau if args.rr_period else tune_m.get("tau", 0.0)
    handles = {}

    def handle(C):
        if C not in handles:
            handles[C] = pkg.from_system(s, device=dev, slice_rows=C,
                                         block_threads=args.block_threads,
                                         blocks_per_sm=args.blocks_per_sm, staging=args.staging)
        return handles[C]

    A = handle(tune_m["slice_rows"])
    b = torch.as_tensor(s.b, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(call, steps, warmup):
        for _ in range(warmup):
            x.zero_()
            call()
        torch.cuda.synchronize(dev)
        times, outs = [], []
        for _ in range(steps):
            x.zero_()
            flush.fill_(1.0)                       # evict the previous step from L2
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = call()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
            outs.append(out)
        return times, outs

    def mixed():
        _, st, it, rr = pkg.pipecg_solve(A, b, x, tol=TOL, precision="mixed", rr_period=rr_m,
                                         tau=tau_m)
        return st, it, rr, A.stats()["replacements"]

    def mixed_deflated():
        _, st, it, rr = pkg.pipecg_solve(A, b, x, tol=TOL, precision="mixed", rr_period=rr_m,
                                         tau=tau_m, deflate=True)
        return st, it, rr, A.stats()["replacements"]

    A_pcg = A_pipe = A
    if not args.skip_fp64:
        A_pcg = handle(autotune.tune_single(s, "pcg", tol=TOL, slice_rows=cands)["slice_rows"])
        A_pipe = handle(autotune.tune_single(s, "fp64", tol=TOL, slice_rows=cands)["slice_rows"])

    def pcg64():
        _, st, it, rr = pkg.pcg_solve(A_pcg, b, x, tol=TOL)
        return st, it, rr, A_pcg.stats()["replacements"]

    def pipe64():
        _, st, it, rr = pkg.pipecg_solve(A_pipe, b, x, tol=TOL, precision="fp64")
        return st, it, rr, A_pipe.stats()["replacements"]

    barrier(dist)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t_mixed, o_mixed = timed(mixed, args.steps, args.warmup)
    torch.cuda.synchronize(dev)
    barrier(dist)
    x_mixed = x.cpu().numpy()
    total = job_seconds(sum(t_mixed), dist, dev)
    st, it, rr, reps = o_mixed[-1]
    grid = A.stats()
    step_s = total / args.steps
    hbm, peak_kind = peaks()
    col_bytes = 2 if (A.info()["col16"] and grid["staged"]) else 4
    alg_bytes = bytes_mixed(n, F, it, reps, col_bytes)
    achieved = alg_bytes / statistics.median(t_mixed) / 1e9
    alg_pre = bytes_mixed_preconditioned(n, F, it, reps)
    achieved_pre = alg_pre / statistics.median(t_mixed) / 1e9
    prof = profiled_traffic(A.info()["slice_rows"])
    traffic = None
    if prof is not None and prof[1] == it:
        traffic = prof[0]

    extra = {}
    def timed_generic(call, steps, warmup, prep=None):
        for _ in range(warmup):
            if prep:
                prep()
            call()
        torch.cuda.synchronize(dev)
        times = []
        for _ in range(steps):
            if prep:
                prep()
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
        return times

    solutions = {"mixed": x_mixed}
    if not args.skip_fp64:
        t_defl, o_defl = timed(mixed_deflated, max(2, args.steps // 2), 1)
        solutions["mixed_deflated"] = x.cpu().numpy()
        t_pcg, o_pcg = timed(pcg64, max(2, args.steps // 2), 1)
        solutions["fp64_pcg"] = x.cpu().numpy()
        t_pipe, o_pipe = timed(pipe64, max(2, args.steps // 2), 1)
        solutions["fp64_pipecg"] = x.cpu().numpy()
        dgemm = fp64_dgemm_tflops(dev)
        pst, pit, prr, preps = o_pcg[-1]
        qst, qit, qrr, qreps = o_pipe[-1]
        mp = statistics.median(t_pcg)
        mq = statistics.median(t_pipe)
        dst, dit, drr, dreps = o_defl[-1]
        extra = {
            "mixed_deflated": {"s": statistics.median(t_defl), "iters": dit, "relres": drr,
                               "status": dst, "replacements": dreps},
            "fp64_pcg": {"s": mp, "iters": pit, "relres": prr, "status": pst,
                         "slice_rows": A_pcg.info()["slice_rows"],
                         "alg_gbs": bytes_pcg64(n, F, pit, preps) / mp / 1e9,
                         "fp64_tflops": 2.0 * PCG64_FP64_INSTR_PER_CELL * n * pit / mp / 1e12,
                         "frac_fp64_dgemm": 2.0 * PCG64_FP64_INSTR_PER_CELL * n * pit / mp
                         / 1e12 / dgemm},
            "fp64_peak": {"dgemm_tflops": dgemm,
                          "how": "torch.matmul float64 4096^3 (cuBLAS), 2 n^3 flops, best of 5, "
                                 "CUDA events; FP64 solvers count 2 flops per FP64 FMA"},
            "fp64_pipecg": {"s": mq, "iters": qit, "relres": qrr, "status": qst,
                            "slice_rows": A_pipe.info()["slice_rows"],
                            "alg_gbs": bytes_pipe64(n, F, qit, qreps) / mq / 1e9},
            "speedup_mixed_vs_fp64_pcg": mp / statistics.median(t_mixed),
        }

    # end to end through the public API: pinned host b in, solve, x back to pinned host
    hb = torch.empty(n, dtype=torch.float64).pin_memory()
    hb.copy_(torch.as_tensor(s.b))
    hx = torch.empty(n, dtype=torch.float64).pin_memory()
    bd = torch.empty(n, dtype=torch.float64, device=dev)

    def e2e_step():
        bd.copy_(hb, non_blocking=True)
        x.zero_()
        pkg.pipecg_solve(A, bd, x, tol=TOL, precision="mixed", rr_period=rr_m, tau=tau_m)
        hx.copy_(x, non_blocking=True)
        return None

    t_e2e, _ = timed(e2e_step, args.steps, 1)
    e2e_s = job_seconds(statistics.mean(t_e2e), dist, dev)

    batched = batched_x = piso_x = None
    if not args.skip_batched:
        batched, batched_x = run_batched(args, dev, pkg, timed_fn=timed_generic)
    pressure = autograd_case = heat = amg_case = piso_case = None
    if not args.skip_extra:
        amg_case, amg_x = run_amg(args, dev, pkg, s, timed_fn=timed_generic)
        solutions.update(amg_x)
        piso_case, piso_x = run_piso(args, dev, pkg, timed_fn=timed_generic)
        pressure = run_pressure(args, dev, pkg, timed_fn=timed_generic)
        autograd_case = run_autograd(args, dev, pkg, timed_fn=timed_generic)
        heat = run_heat(args, dev, pkg, timed_fn=timed_generic)

    # CPU baseline: the oracle on this host, one complete solve, rank 0 only
    cpu = cpu_omp = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        import oracle
        t1, r1 = oracle_solve(s, omp=False)
        cpu = {"value": t1, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"one complete FP64 Jacobi-PCG solve of the {args.size}^3 case to 1e-8 "
                         f"({r1.iters} iterations; plain C oracle, one host core)"}
        t2, r2 = oracle_solve(s, omp=True)
        cpu_omp = {"value": t2, "unit": "s", "cores": oracle.threads(omp=True), "kind": "oracle",
                   "sample": f"the same solve ({r2.iters} iterations) by the oracle's C source "
                             f"built with OpenMP, all host threads"}

    relres_oracle = accuracy = None
    if rank == 0:
        import oracle
        relres_oracle = oracle.true_relres(s, x_mixed)
        if not args.skip_accuracy:
            accuracy = accuracy_report(s, solutions, batched_x, piso_x)
            errs = accuracy["errors"]
            for key, leg in (("mixed_deflated", extra.get("mixed_deflated")),
                             ("fp64_pcg", extra.get("fp64_pcg")),
                             ("fp64_pipecg", extra.get("fp64_pipecg"))):
                if leg is not None and key in errs:
                    leg["error_vs_fp64"] = errs[key]
            if batched is not None:
                batched["error_vs_fp64_max"] = errs.get("batched_max")
            if amg_case is not None:
                for prec in ("mixed", "fp64", "pipelined_fp64"):
                    amg_case[prec]["error_vs_fp64"] = errs.get("amg_" + prec)
            if piso_case is not None:
                piso_case["error_vs_fp64_last_step"] = errs.get("piso_pressure_last_step")
            if pressure is not None:
                pressure["error_vs_fp64"] = None
                pressure["error_note"] = ("no oracle reference at 256^3: its tight FP64 solve "
                                          "takes minutes on the host")

    line = {
        "metric": METRIC, "value": step_s, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(size=args.size),
                   "solver": "mixed pipelined Jacobi-PCG (libldupcg, k_mixed)",
                   "cells": n, "faces": F, "slice_rows": A.info()["slice_rows"],
                   "blocks_per_sm": args.blocks_per_sm, "staging": args.staging,
                   "grid_blocks": grid["grid_blocks"], "block_threads": grid["block_threads"],
                   "rr_period": rr_m, "tau": tau_m, "l2": "256 MB flush before every step",
                   "parallelism": "replicas" if world > 1 else "single"},
        "solve": {"status": st, "iters": it, "replacements": reps, "relres": rr,
                  "relres_oracle": relres_oracle,
                  "error_vs_fp64": accuracy["errors"]["mixed"] if accuracy else None},
        "roofline": {"bound": "hbm", "achieved": achieved_pre, "peak": hbm, "unit": "GB/s",
                     "frac": achieved_pre / hbm, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "k_mixed (persistent, one launch per solve)",
                     "alg_bytes_per_launch": alg_pre,
                     "alg_model": "preconditioned pipelined PCG: (4n+16F+80n) B per float "
                                  "iteration + (8n+24F+24n) B per FP64 residual",
                     "frac_scaled_model": achieved / hbm,
                     "alg_bytes_scaled_model": alg_bytes,
                     "frac_dram": (traffic / statistics.median(t_mixed) / 1e9 / hbm
                                   if traffic else None),
                     "target_fraction": "frac_dram"},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n,
                "step_ms_min_median_max": [min(t_e2e) * 1e3, statistics.median(t_e2e) * 1e3,
                                           max(t_e2e) * 1e3]},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "cpu_baseline_omp": cpu_omp,
        "accuracy": accuracy,
        "batched": batched,
        "pressure256": pressure,
        "differentiable": autograd_case,
        "heat_steps": heat,
        "amg_pcg": amg_case,
        "piso_pressure": piso_case,
    }
    line.update(extra)
    emit(line, ranks)
    for h in handles.values():
        h.close()
    if dist is not None:
        dist.destroy_process_group()


def run_batched(args, dev, pkg, timed_fn):
    """512 uneven systems (cube sides uniform in 8..48), mixed precision to
    1e-8: one persistent launch (autotuned layout and teams) against the same
    solves as 512 separate calls."""
    import numpy as np
    import torch

    import ldu_cases as lc
    from paper_1505_07630_gb300 import autotune

    systems = lc.config4(nsys=args.batch_systems)
    rr_b = args.rr_period or 12
    best = autotune.tune_batched(systems, tol=TOL, rr_period=rr_b)
    A = pkg.from_systems(systems, device=dev, slice_rows=best["slice_rows"])
    pkg.ldu_batch_schedule(A, max_team=best["max_team"], team_work_scale=best["team_work_scale"])
    b = torch.as_tensor(np.concatenate([s.b for s in systems]), device=dev)
    x = torch.zeros_like(b)

    def one_launch():
        pkg.pcg_solve_batched(A, b, x, tol=TOL, precision="mixed", rr_period=rr_b)

    t_batch = timed_fn(one_launch, max(2, args.steps // 2), 1, prep=x.zero_)
    worst, its, rrs, sts = pkg.ldu_batch_results(A)
    info = pkg.ldu_batch_info(A)
    # the same solves, one call per system (handles built outside the timing)
    offs = np.concatenate([[0], np.cumsum([s.n for s in systems])])
    handles = [pkg.from_system(s, device=dev, slice_rows=best["slice_rows"]) for s in systems]
    views = [(b[offs[k]:offs[k + 1]], x[offs[k]:offs[k + 1]]) for k in range(len(systems))]

    def separate():
        for Ak, (bk, xk) in zip(handles, views):
            pkg.pipecg_solve(Ak, bk, xk, tol=TOL, precision="mixed", rr_period=rr_b)

    t_sep = timed_fn(separate, 1, 1, prep=x.zero_)
    for Ak in handles:
        Ak.close()
    staged_b = int(A.stats()["staged"])
    cb = 2 if (A.info()["col16"] and staged_b) else 4
    alg = sum(bytes_mixed(s.n, s.nfaces, int(its[k]), int(its[k]) // rr_b + 2, cb)
              for k, s in enumerate(systems))
    tb = statistics.median(t_batch)
    xh = x.cpu().numpy()
    A.close()
    return {"systems": len(systems), "cells": int(offs[-1]), "one_launch_s": tb,
            "separate_calls_s": statistics.median(t_sep), "speedup": statistics.median(t_sep) / tb,
            "worst_status": int(worst), "max_iters": int(its.max()), "mean_iters": float(its.mean()),
            "max_relres": float(rrs.max()), "alg_gbs": alg / tb / 1e9,
            "tuned": {k: best[k] for k in ("slice_rows", "max_team", "team_work_scale")},
            "grid_blocks": info["grid_blocks"], "teams_max": info["max_team"],
            "staged": staged_b,
            "ntasks": info["ntasks"]}, (systems, xh)


def run_amg(args, dev, pkg, s, timed_fn):
    """Aggregation-AMG preconditioned CG (Sec. 5, Table 2's AMG-CG) on the
    headline system to 1e-8: hierarchy setup (device kernels, once per matrix), one
    V-cycle in each precision, and the whole solve with the FP64 cycle and
    with the float cycle inside the FP64 outer CG."""
    import time

    import torch

    pkg.amg_from_system(s, device=dev).close()   # warm-up: module load, memory pool
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    M = pkg.amg_from_system(s, device=dev)
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t0
    b = torch.as_tensor(s.b, device=dev)
    x = torch.zeros_like(b)
    z = torch.empty_like(b)
    b32 = b.float()
    z32 = torch.empty_like(b32)
    out = {"setup_s": setup_s, "levels": M.info()["rows"]}
    for name, bb, zz in (("vcycle_fp64_ms", b, z), ("vcycle_fp32_ms", b32, z32)):
        def cycles(bb=bb, zz=zz):
            for _ in range(10):
                pkg.ldu_amg_vcycle(M, bb, zz)
        out[name] = statistics.median(timed_fn(cycles, 3, 1)) * 100.0
    xs = {}
    for prec in ("mixed", "fp64", "pipelined_fp64"):
        res = {}

        def solve(prec=prec, res=res):
            if prec == "pipelined_fp64":
                res["out"] = pkg.amg_pipecg_solve(M, b, x, tol=TOL, maxit=500)
            else:
                res["out"] = pkg.amg_pcg_solve(M, b, x, tol=TOL, maxit=500, precision=prec)

        t = timed_fn(solve, 3, 1, prep=x.zero_)
        _, it, rr, st = res["out"]
        out[prec] = {"s": statistics.median(t), "iters": it, "relres": rr, "status": st}
        xs["amg_" + prec] = x.cpu().numpy()
    M.close()
    return out, xs


def run_spmv(pkg, A, nfaces, dev, reps=20, rounds=5):
    """ldu_spmv (Sec. 2.1's product, Table 1's first kernel) alone, FP32 and
    FP64, on a system whose product data is several times the 129 MB L2: the
    L2 is flushed once, then `reps` back-to-back products are timed between
    two CUDA events (the median of `rounds`); a flush before every launch
    would leave its own write-back of dirty lines inside a product this
    short.  Algorithmic bytes per product: x in and y out (T each), the
    scaling factor sd (8 B) per row, and an int32 column and a value per
    stored off-diagonal entry (2F entries, padding excluded)."""
    import torch

    n = A.n
    hbm, _ = peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {"cells": n, "faces": nfaces, "launches_per_timing": reps,
           "timing": "L2 flushed once, back-to-back products between CUDA events"}
    for prec, dt, tb in (("fp32", torch.float32, 4), ("fp64", torch.float64, 8)):
        xv = torch.rand(n, dtype=dt, device=dev)
        yv = torch.empty_like(xv)
        for _ in range(3):
            pkg.ldu_spmv(A, xv, yv, precision=prec)
        per = []
        for _ in range(rounds):
            flush.fill_(1.0)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                pkg.ldu_spmv(A, xv, yv, precision=prec)
            e1.record(stream)
            e1.synchronize()
            per.append(e0.elapsed_time(e1) * 1e-3 / reps)
        t = statistics.median(per)
        alg = n * (2 * tb + 8) + 2 * nfaces * (4 + tb)
        out[prec] = {"us": t * 1e6, "alg_bytes": alg, "gbs": alg / t / 1e9,
                     "frac": alg / t / 1e9 / hbm}
    return out


def run_pressure(args, dev, pkg, timed_fn):
    """The icoFoam-style pressure system on a graded 256³ box (pure Neumann,
    one pinned cell): mixed pipelined PCG with constant-vector deflation
    against FP64 Jacobi-PCG, both to 1e-8, slice height 128."""
    import torch

    import ldu_cases as lc

    s = lc.config3(s=256, seed=0)
    A = pkg.from_system(s, device=dev, slice_rows=128)
    b = torch.as_tensor(s.b, device=dev)
    x = torch.zeros_like(b)
    out = {"cells": s.n, "faces": s.nfaces}

    def mixed():
        pkg.pipecg_solve(A, b, x, tol=TOL, maxit=50000, precision="mixed", deflate=True)

    def pcg():
        pkg.pcg_solve(A, b, x, tol=TOL, maxit=50000)

    hbm, _ = peaks()
    cb = 2 if A.info()["col16"] else 4
    for name, call in (("mixed_deflated", mixed), ("fp64_pcg", pcg)):
        t = timed_fn(call, 2, 1, prep=x.zero_)
        st = A.stats()
        ts = statistics.median(t)
        out[name] = {"s": ts, "iters": st["iters"],
                     "replacements": st["replacements"], "relres": st["relres"],
                     "status": st["status"]}
        # the vectors (0.7 GB in float) no longer fit the L2 here: the
        # algorithmic bytes are what has to come from HBM
        alg = (bytes_mixed(s.n, s.nfaces, st["iters"], st["replacements"], cb, deflated=True)
               if name == "mixed_deflated" else
               bytes_pcg64(s.n, s.nfaces, st["iters"], st["replacements"]))
        out[name].update(alg_bytes=alg, alg_gbs=alg / ts / 1e9, frac=alg / ts / 1e9 / hbm)
    out["speedup_mixed_vs_fp64_pcg"] = out["fp64_pcg"]["s"] / out["mixed_deflated"]["s"]
    out["spmv"] = run_spmv(pkg, A, s.nfaces, dev)
    A.close()
    return out


def run_heat(args, dev, pkg, timed_fn):
    """laplacianFoam-style transient: 10 backward-Euler steps of the 128³
    lognormal diffusion system, dt = h² (mass h³/dt per cell), from a smooth
    initial field, each step a mixed solve to 1e-8 warm-started from the
    last, on one handle."""
    import numpy as np
    import torch

    import ldu_cases as lc

    s = lc.config2(s=args.size, seed=0)
    h = 1.0 / args.size
    mass = np.full(s.n, h ** 3 / (1.0 * h * h))
    A = pkg.ldu_create(s.n, *(torch.as_tensor(a, device=dev) for a in
                              (s.owner, s.neighbour, s.diag + mass, s.upper, s.lower)),
                       slice_rows=128)
    m = torch.as_tensor(mass, device=dev)
    # a smooth initial temperature, sin(pi x) sin(pi y) sin(pi z) at the cell centres
    nx = args.size
    c = np.asarray(s.cell_of)
    ci, cj, ck = c % nx, (c // nx) % nx, c // (nx * nx)
    T0 = torch.as_tensor(np.sin(np.pi * (ci + 0.5) / nx) * np.sin(np.pi * (cj + 0.5) / nx)
                         * np.sin(np.pi * (ck + 0.5) / nx), device=dev)
    T = T0.clone()
    out = {}

    def steps():
        T.copy_(T0)
        _, st, its, rr = pkg.ldu_heat_steps(A, m, T, 10, tol=TOL, precision="mixed")
        out.update(status=st, iterations=its, relres_last=rr)

    t = timed_fn(steps, 2, 1)
    A.close()
    return {"cells": s.n, "steps": 10, "dt_over_h2": 1.0, "s_per_step": statistics.median(t) / 10,
            "iterations_per_step": out["iterations"] / 10, "relres_last": out["relres_last"],
            "status": out["status"]}


def run_piso(args, dev, pkg, timed_fn):
    """icoFoam-style pressure stages (Sec. 2's PISO): 10 time steps on the
    graded 128³ pressure system (pure Neumann with a pinned cell), predicted
    fluxes phi*_k = phi_0 + 1e-3 k dphi, each step b = -div(phi*), a mixed
    deflated solve to 1e-8 warm-started from the previous pressure, and the
    flux correction, on one handle."""
    import torch

    import ldu_cases as lc
    from ldu_cases import rng

    s = lc.config3(s=args.size, seed=0)
    A = pkg.from_system(s, device=dev, slice_rows=128)
    coef = torch.as_tensor(s.coef, device=dev)
    phi0 = torch.as_tensor(rng.uniform(rng.stream_base(0, "piso-flux"), s.nfaces, -1.0, 1.0),
                           device=dev)
    dphi = torch.as_tensor(rng.uniform(rng.stream_base(0, "piso-dflux"), s.nfaces, -1.0, 1.0),
                           device=dev)
    phi = torch.empty_like(phi0)
    p = torch.zeros(s.n, dtype=torch.float64, device=dev)
    out = {"iters": 0}

    def steps():
        p.zero_()
        out["iters"] = 0
        for k in range(10):
            torch.add(phi0, dphi, alpha=1e-3 * k, out=phi)
            st, it, rr = pkg.ldu_piso_pressure(A, coef, phi, p, tol=TOL, precision="mixed",
                                               deflate=True)
            out["iters"] += it
            out["status"], out["relres"] = st, rr

    t = timed_fn(steps, 2, 1)
    A.close()
    # the last step's system, for the error against the oracle: b = -div(phi*_9)
    from oracle import piso as opiso
    phi9 = torch.add(phi0, dphi, alpha=1e-3 * 9).cpu().numpy()   # the step's own input
    b9 = -opiso.divergence_fast(s.owner, s.neighbour, s.n, phi9)
    return ({"cells": s.n, "faces": s.nfaces, "steps": 10, "s_per_step": statistics.median(t) / 10,
             "iterations_per_step": out["iters"] / 10, "relres_last": out["relres"],
             "status": out["status"]}, (s, b9, p.cpu().numpy()))


def run_autograd(args, dev, pkg, timed_fn):
    """Differentiable solve on a 64³ mesh, batch of 8 diffusivity fields:
    loss 0.5 ||x(c) - x_t||², forward solve plus backward (adjoint solve and
    face/diagonal/RHS gradients) in one batched handle, mixed precision to
    1e-10; targets from FP64 solves of the reference fields.  Timed again
    with the cell diffusivities as the parameters."""
    import numpy as np
    import torch

    import ldu_cases as lc

    systems, refs = lc.config5()
    Ar = pkg.from_systems(refs, device=dev)
    br = torch.as_tensor(np.concatenate([r.b for r in refs]), device=dev)
    xt, *_ = pkg.pcg_solve_batched(Ar, br, tol=1e-12, precision="fp64")
    Ar.close()
    A = pkg.from_systems(systems, device=dev)
    cat = lambda name: torch.as_tensor(np.concatenate([getattr(q, name) for q in systems]),  # noqa: E731
                                       device=dev)
    coef, extra, b = cat("coef"), cat("diag_extra"), cat("b")

    def step():
        c = coef.clone().requires_grad_(True)
        bb = b.clone().requires_grad_(True)
        xs = pkg.ldu_solve(A, c, extra, bb, precision="mixed", tol=1e-10)
        loss = 0.5 * ((xs - xt) ** 2).sum()
        loss.backward()
        return c.grad

    t = timed_fn(step, 2, 1)
    # the same loss as a function of every cell's diffusivity (harmonic-mean
    # faces and wall terms in the library's kernels)
    kc = torch.as_tensor(np.concatenate([q.meta["k_cell"] for q in systems]), device=dev)
    gf = torch.as_tensor(np.concatenate([q.meta["g_face"] for q in systems]), device=dev)
    bf = torch.as_tensor(np.concatenate([q.meta["bfac"] for q in systems]), device=dev)

    def step_k():
        kk = kc.clone().requires_grad_(True)
        c, e = pkg.harmonic_coeffs(A, kk, gf, bf)
        xs = pkg.ldu_solve(A, c, e, b, precision="mixed", tol=1e-10)
        (0.5 * ((xs - xt) ** 2).sum()).backward()
        return kk.grad

    t_k = timed_fn(step_k, 2, 1)
    A.close()
    return {"systems": len(systems), "cells_each": systems[0].n,
            "faces_each": systems[0].nfaces, "forward_backward_s": statistics.median(t),
            "forward_backward_cell_k_s": statistics.median(t_k)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--slice-rows", type=int, default=0)
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--staging", type=int, default=0, choices=[0, -1])
    ap.add_argument("--rr-period", type=int, default=0)
    ap.add_argument("--tau", type=float, default=0.0)
    ap.add_argument("--skip-accuracy", action="store_true",
                    help="skip the errors against the oracle's tight solution")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-extra", action="store_true",
                    help="skip the 256^3 pressure and differentiable-solve timings")
    ap.add_argument("--batch-systems", type=int, default=512)
    ap.add_argument("--print-digest", action="store_true")
    args = ap.parse_args()
    if args.print_digest:
        print(source_digest())
        return
    if args.warmup < 0 or args.steps < 1:
        ap.error("need steps >= 1")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
