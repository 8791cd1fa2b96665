"""Benchmark: RHS solves per second of the mixed-precision DDM-preconditioned solver.

Workload (default, the largest 2D configuration): two-layer medium (c = 1 below y = 0.37, 1.5
above, the interface between grid lines and not on a subdomain boundary), omega = 2 pi 50,
1024^2 interior grid (h = 1/1024), 16x16 subdomains of 64^2 with a 12-cell PML (quadratic,
strength 30), 64 right-hand sides, each a unit-mass Gaussian (width 2h) at a seeded uniform
position; complex64 sweeps (3xTF32 tensor-core substitutions) + FP64 FGMRES to 1e-6 with two DDM
rounds per preconditioner application.  One step = one dds_solve of the whole 64-RHS batch (every
RHS must also reach relative L2 error <= 1e-6 against the plain FP64 GPU solve, checked after
timing).  Other workloads: --workload const2d_640 | const3d_128 | table5 | serve.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload NAME]

N > 1 runs one independent replica per GPU (RHS sharding, no collective on the data path);
value is the whole-job RHS/s over all ranks.  Rank 0 prints one JSON line; the accuracy, FP64
comparator and latency keys come last.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RHS solves/sec at rel. L2 1e-6 vs plain FP64 GPU sweep; p50/p99 latency"
WORKLOAD = "layer2d_1024"
WORKLOADS = {
    "layer2d_1024": ("2D two-layer medium (c=1 for y<0.37, c=1.5 above; interface not aligned to "
                     "subdomain boundaries), k=2*pi*50, 1024x1024 grid, 16x16 subdomains (64x64 + "
                     "12-cell PML), 64 RHS seeded Gaussian point sources (width 2h), DDM (3 rounds) "
                     "as FGMRES preconditioner, tol 1e-6, complex64 sweeps / FP64 factorisation "
                     "and FGMRES"),
    "const2d_640": ("2D constant medium c=1, k=2*pi*40, 640x640 interior grid, 8x8 subdomains "
                    "(80x80 + 12-cell PML), 16 RHS Gaussian point sources (width 2h) at seeded "
                    "uniform positions, complex64 sweeps + FP64 FGMRES to 1e-6 (2 rounds)"),
    "const3d_128": ("3D constant medium c=1, k=2*pi*10, 128^3 grid, 7-point FD, 4x4x4 subdomains "
                    "(32^3 + 8-cell PML), 8 RHS seeded Gaussian point sources, 8 diagonal sweeps, "
                    "complex64 substitutions with FP64 FGMRES refinement to 1e-6"),
    "const2d_128": ("2D constant medium c=1 on the unit square, k=2*pi*8, 128x128 interior grid, "
                    "16-cell PML, 2x2 subdomains, one Gaussian point source (width 2h) at "
                    "(0.5,0.5)"),
}


def workload_desc(name: str) -> str:
    if name in WORKLOADS:
        return WORKLOADS[name]
    if name.startswith("table5_"):
        N = int(name.split("_")[1])
        return (f"2D constant medium, {300 * N}x{300 * N} grid, {N}x{N} subdomains of 300^2 "
                f"(30-point PML), four approximated delta sources (Eq. 5.4), one RHS")
    return name


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.path is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _reduce_max(value: float, world: int):
    """Max over ranks (the slowest replica sets the whole job's time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, rhs_per_rank: int, steps: int, max_seconds: float):
    """Replicas: every rank solves rhs_per_rank right-hand sides per step; the job's rate is all
    ranks' right-hand sides over the slowest rank's time."""
    return world * rhs_per_rank * steps / max_seconds if max_seconds > 0 else None


def _barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------------------
# CPU oracle (the "reference" arm and the cpu_baseline)
# ------------------------------------------------------------------------------------------
_ORACLE_CACHE = {}


def _oracle_setup(wl):
    """The oracle's problem, assembled global operator and factored local problems of a
    workload (set-up, kept across samples and outside their timing)."""
    from oracle.discretize import Problem, assemble_global
    from oracle.sweep import LocalProblems
    key = id(wl)
    if key not in _ORACLE_CACHE:
        prob = Problem(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength)
        A, _ = assemble_global(prob)
        _ORACLE_CACHE.clear()
        _ORACLE_CACHE[key] = (wl, prob, A, LocalProblems(prob))
    return _ORACLE_CACHE[key][1:]


def oracle_solve_sample(wl, rhs_index: int, workers: int, tol: float):
    """One FGMRES solve of one right-hand side of the workload by the CPU oracle."""
    from oracle.discretize import extend_interior, rhs_from_source
    from oracle.fgmres import fgmres
    from oracle.sweep import ddm_solve
    prob, A, loc = _oracle_setup(wl)
    b = rhs_from_source(prob, extend_interior(prob, wl.f[rhs_index]))
    shape = b.shape
    t0 = time.perf_counter()
    x, it, hist = fgmres(lambda v: A @ v,
                         lambda v: ddm_solve(prob, v.reshape(shape), wl.rounds, loc,
                                             workers=workers).ravel(),
                         b.ravel(), tol=tol, maxit=60)
    return time.perf_counter() - t0, it, hist[-1]


def cpu_baseline_sample(wl, tol, budget_s: float = 10.0):
    """The CPU oracle on right-hand sides of the workload, one after another, until about
    budget_s seconds of work (at least one solve)."""
    workers = os.cpu_count() or 1
    total, done, its = 0.0, 0, []
    while done < wl.f.shape[0] and (done == 0 or total < budget_s):
        dt, it_o, _ = oracle_solve_sample(wl, done, workers, tol)
        total += dt
        done += 1
        its.append(it_o)
    return {"value": done / total, "unit": "RHS/s", "cores": workers, "kind": "oracle",
            "sample": f"FGMRES solves (tol {tol:g}, {min(its)}-{max(its)} iterations) of "
                      f"right-hand sides 0..{done - 1} of the same workload, {total:.1f} s"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2003_02585_gb300 import synth
    wl = synth.workload(args.workload)
    workers = os.cpu_count() or 1
    for w in range(args.warmup):
        oracle_solve_sample(wl, w % wl.f.shape[0], workers, args.tol)
    times = []
    iters = []
    for k in range(args.steps):
        dt, it, _ = oracle_solve_sample(wl, k % wl.f.shape[0], workers, args.tol)
        times.append(dt)
        iters.append(it)
    total = sum(times)
    value = args.steps / total
    sample = (f"one FGMRES solve (tol {args.tol:g}) of one of the {wl.f.shape[0]} right-hand "
              f"sides per step, oracle subdomain solves of each sweep step on a thread pool")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload), "name": args.workload,
                   "rhs_per_step": 1},
        "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": workers, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "fgmres_iterations": iters,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def fp64_check(args, wl, R, f_dev, u_mixed, stream, flush):
    """Relative L2 error of the mixed solve against the plain FP64 GPU solve (tol 1e-10), and
    the FP64 path's own throughput at the benchmark tolerance, timed with the mixed arm's
    protocol: the same warm-up count, timed steps (--fp64-steps, default --steps) and L2 flush
    between steps, CUDA events on the same stream."""
    import torch

    from paper_2003_02585_gb300 import dds

    ctx64 = dds.Context(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength,
                        precision="fp64", plan=args.plan)
    u64, it64, rel64 = ctx64.solve(f_dev, tol=1e-10, maxit=args.maxit, rounds=wl.rounds)
    torch.cuda.synchronize()
    err = [float(torch.linalg.vector_norm(u_mixed[r] - u64[r]) / torch.linalg.vector_norm(u64[r]))
           for r in range(R)]
    steps = args.steps if args.fp64_steps is None else args.fp64_steps
    fp64_warm = args.warmup if args.fp64_warmup is None else args.fp64_warmup
    for _ in range(fp64_warm if steps > 0 else 0):
        ctx64.solve(f_dev, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)
    torch.cuda.synchronize()
    fp64_ms, its = [], []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, it_c, rel_c = ctx64.solve(f_dev, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)
        e1.record(stream)
        e1.synchronize()
        fp64_ms.append(e0.elapsed_time(e1))
        its.append(it_c)
    fp64_value = R * len(fp64_ms) / (sum(fp64_ms) / 1e3) if fp64_ms else None
    ctx64.close()
    del ctx64
    spread = ({"ms_min": min(fp64_ms), "ms_median": statistics.median(fp64_ms),
               "ms_max": max(fp64_ms)} if fp64_ms else None)
    return err, fp64_ms, fp64_value, u64, spread, sorted(set(its))


def time_variant(args, wl, R, f_dev, stream, flush, precision, u64):
    """The same timed solve loop for another single-precision sweep variant (same workload,
    steps, L2 flush), with its accuracy against the FP64 GPU solve."""
    import torch

    from paper_2003_02585_gb300 import dds

    ctx = dds.Context(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength,
                      precision=precision, plan=args.plan)
    if not args.no_autotune:
        ctx.autotune(R, wl.rounds)
    its = []
    for _ in range(args.warmup):
        ctx.solve(f_dev, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u, it, _ = ctx.solve(f_dev, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        its.append(it)
    err = None
    if u64 is not None:
        err = max(float(torch.linalg.vector_norm(u[r] - u64[r]) / torch.linalg.vector_norm(u64[r]))
                  for r in range(R))
    ctx.close()
    return {"precision": precision, "dtype": DTYPE[precision],
            "value": R * len(ms) / (sum(ms) / 1e3), "unit": "RHS/s",
            "ms_per_step": sum(ms) / len(ms), "max_rel_l2_vs_fp64_gpu": err,
            "fgmres_iterations": sorted(set(its))}

def short_measure(args, name, stream, flush):
    """A shorter measurement of another workload, reported beside the headline: the same solve
    loop (warm-up, --also-steps timed steps, L2 flush, CUDA events), its FGMRES iterations and,
    for 2D workloads, its error against the FP64 GPU solve and that solve's rate."""
    import torch

    from paper_2003_02585_gb300 import dds, synth

    wl = synth.workload(name)
    R = wl.f.shape[0]
    ctx = dds.Context(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength,
                      precision=args.precision, plan=args.plan)
    if not args.no_autotune and len(wl.n) == 2:
        ctx.autotune(R, wl.rounds)
    f_dev = torch.from_numpy(ctx.extend(wl.f)).to(flush.device)

    def timed(c, steps):
        ms, its = [], []
        for _ in range(args.warmup):
            c.solve(f_dev, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            u, it, _ = c.solve(f_dev, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            its.append(it)
        return u, ms, its

    u, ms, its = timed(ctx, args.also_steps)
    out = {"workload": workload_desc(name), "name": name, "value": R * len(ms) / (sum(ms) / 1e3),
           "unit": "RHS/s", "ms_per_step": sum(ms) / len(ms), "steps": len(ms),
           "fgmres_iterations": sorted(set(its)), "setup_seconds": ctx.info()["setup_seconds"]}
    if name.startswith("table5_"):
        N = int(name.split("_")[1])
        out["paper"] = {"fgmres_iterations": TABLE5_PAPER[N][0], "solve_s": TABLE5_PAPER[N][1],
                        "hardware": "the paper's CPU cluster, one core per subdomain"}
    ctx.close()
    if len(wl.n) == 2 and not args.no_fp64:
        c64 = dds.Context(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength,
                          precision="fp64", plan=args.plan)
        u64, _, _ = c64.solve(f_dev, tol=1e-10, maxit=args.maxit, rounds=wl.rounds)
        out["max_rel_l2_vs_fp64_gpu"] = max(
            float(torch.linalg.vector_norm(u[r] - u64[r]) / torch.linalg.vector_norm(u64[r]))
            for r in range(R))
        del u64
        _, ms64, _ = timed(c64, args.also_steps)
        out["fp64_comparator"] = {"value": R * len(ms64) / (sum(ms64) / 1e3), "unit": "RHS/s",
                                  "steps": len(ms64)}
        c64.close()
    del f_dev
    torch.cuda.empty_cache()
    return out


def run_gpu(args):
    import torch

    from paper_2003_02585_gb300 import build as lbuild
    from paper_2003_02585_gb300 import dds, synth

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lbuild.build()
    wl = synth.workload(args.workload, args.nrhs)
    if args.rounds is not None:
        wl.rounds = args.rounds
    R = wl.f.shape[0]

    ctx = dds.Context(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength,
                      precision=args.precision, plan=args.plan)
    # launch shapes picked by measurement on this workload (set-up work, outside the timing), or
    # pinned by --shape (panel width, panels per CTA, trace kernel)
    tuned = None
    if args.shape:
        pw, npc, tk = (int(v) for v in args.shape.split(","))
        ctx.set_launch_shape(pw, npc, tk)
        tuned = {"panel_width": pw, "panels_per_cta": npc, "trace_ctas_per_sm": tk, "table": []}
    elif not args.no_autotune:
        tuned = ctx.autotune(R, wl.rounds)
    info = ctx.info()
    f_host = ctx.extend(wl.f)
    f_dev = torch.from_numpy(f_host).to(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > 129 MB L2

    iters_seen = []
    for _ in range(args.warmup):
        u, it, rel = ctx.solve(f_dev, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)
        iters_seen.append(it)
    torch.cuda.synchronize()

    launches0 = ctx.launches()
    step_ms = []
    with ClockSampler(local) as clk:
        _barrier(world)
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.fill_(1)                                    # L2 flush between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            u, it, rel = ctx.solve(f_dev, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            iters_seen.append(it)
        torch.cuda.synchronize()
        _barrier(world)
    clocks = clk.summary()
    launches = ctx.launches() - launches0
    total_ms = _reduce_max(sum(step_ms), world)
    value = whole_job_rate(world, R, args.steps, total_ms / 1e3)
    u_mixed = u

    # end to end through the C ABI with host (pinned) buffers, right after the device-timed steps
    # (before the comparator and variant contexts come and go)
    f_pin = torch.from_numpy(f_host).pin_memory()
    u_pin = torch.empty_like(f_pin).pin_memory()
    fn = f_pin.numpy()
    un = u_pin.numpy()
    e2e_s = []
    # untimed warm-up calls first: the first call through host pointers allocates the library's
    # staging buffers and captures the graph for their addresses
    for _ in range(args.warmup if args.e2e_steps > 0 else 0):
        st = ctx._lib.dds_solve(ctx._h, ctx._ptr(fn), R, ctx._ptr(un), args.tol, args.maxit,
                                wl.rounds, None, None)
        if st not in (0, 4):
            raise RuntimeError(f"dds_solve from host buffers failed: {st}")
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        st = ctx._lib.dds_solve(ctx._h, ctx._ptr(fn), R, ctx._ptr(un), args.tol, args.maxit,
                                wl.rounds, None, None)
        e2e_s.append(time.perf_counter() - t0)
        if st not in (0, 4):
            raise RuntimeError(f"dds_solve from host buffers failed: {st}")
    e2e_total = _reduce_max(sum(e2e_s), world) if e2e_s else 0.0
    e2e_value = whole_job_rate(world, R, len(e2e_s), e2e_total)

    # accuracy against the plain FP64 GPU solve, and that solve's own throughput
    if args.no_fp64:
        err, fp64_ms, fp64_value, u64, fp64_spread, fp64_its = [float("nan")], [], None, None, \
            None, []
    else:
        err, fp64_ms, fp64_value, u64, fp64_spread, fp64_its = fp64_check(
            args, wl, R, f_dev, u_mixed, stream, flush)
    # the other single-precision sweep variants, timed the same way
    variants = [time_variant(args, wl, R, f_dev, stream, flush, p, u64)
                for p in args.variants.split(",")
                if p and p != "none" and p != args.precision]
    del u64

    # roofline of the dominant kernel family, timed with CUDA events on the library's stream
    ctx.profile(True)
    ctx.local_solve_counts(reset=True)
    ddm_apps = 0
    for _ in range(args.profile_steps):
        _, it_p, _ = ctx.solve(f_dev, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)
        ddm_apps += it_p
    stats = ctx.kernel_stats()
    ctx.profile(False)
    # zero-work skipping leaves some local problems unsolved: the substitutions are credited only
    # with the ones they ran
    solved, assembled = ctx.local_solve_counts(reset=True)
    work = list(ctx.work_per_ddm(R, wl.rounds))
    if assembled > 0:
        work[0] *= solved / assembled
    inf = ctx.info()
    geometry = {"plan": inf["plan"], "nrhs": R, "nsub": inf["n_sub"], "T": inf["trace_len"],
                "Nglob": int(np.prod(inf["G"][:len(wl.n)])),
                "Nloc": int(np.prod(inf["M"][:len(wl.n)])),
                "Mb": int(np.prod(inf["M"][:len(wl.n) - 1])),
                "trace_kernel": inf.get("trace_kernel", 1),
                "subst_kernel": inf.get("subst_kernel", 2),
                "sweeps": (2 ** len(wl.n)) * wl.rounds,
                "panel_width": (tuned or {}).get("panel_width"),
                "panels_per_cta": (tuned or {}).get("panels_per_cta")}
    # the dense MMA rate of the piece type on this GPU, next to the recipe's peak (set-up work)
    kind = SPLIT_KIND.get(args.precision, "fp32")
    mma_rate = dds.tensor_rate(kind) if kind in ("tf32", "bf16") and args.profile_steps > 0 else None
    roofline, roofline_kernels = (roofline_entry(stats, work, ddm_apps, args, geometry, mma_rate)
                                  if args.profile_steps > 0 else (None, []))

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_sample(wl, args.tol)

    lat = sorted(step_ms)

    def pct(p):
        return lat[min(len(lat) - 1, int(math.ceil(p / 100.0 * len(lat))) - 1)]

    also = []
    for name in [w for w in args.also.split(",") if w and w != "none" and w != args.workload]:
        also.append(short_measure(args, name, stream, flush))

    # the long, descriptive keys first; the headline evidence (roofline, accuracy, FP64
    # comparator, latency) last, so that a truncated tail of the line still carries it
    line = {
        "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": workload_desc(args.workload), "name": args.workload,
                   "global_batch": R * world, "precision": args.precision,
                   "grid": list(wl.n), "parts": list(wl.parts), "pml_cells": wl.pml_cells,
                   "tol": args.tol, "rounds": wl.rounds, "plan": args.plan,
                   "parallelism": f"replicas x{world} (RHS sharding)",
                   "l2_flush": "256 MB buffer written between timed steps"},
        "roofline_kernels": roofline_kernels,
        "variants": variants,
        "autotune": tuned,
        "other_workloads": also,
        "setup_seconds": info["setup_seconds"],
        "e2e": {"value": e2e_value, "unit": "RHS/s",
                "h2d_bytes_per_step": int(f_host.nbytes), "d2h_bytes_per_step": int(f_host.nbytes)},
        "gpu_launches": launches,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "roofline": roofline,
        "latency_ms": {"p50": pct(50), "p99": pct(99)},
        "accuracy": {"max_rel_l2_vs_fp64_gpu": max(err), "fp64_reference_tol": 1e-10,
                     "fgmres_iterations": sorted(set(iters_seen))},
        "fp64_comparator": {"value": fp64_value, "unit": "RHS/s", "steps": len(fp64_ms),
                            "warmup": (args.warmup if args.fp64_warmup is None else args.fp64_warmup)
                                      if fp64_ms else 0, "spread": fp64_spread,
                            "fgmres_iterations": fp64_its,
                            "what": "same plan, factors and batching in FP64 (plain FP64 GPU "
                                    "sweep + FP64 FGMRES), same timing protocol"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


DTYPE = {"mixed": "c64 sweeps (3xTF32 tensor-core substitutions) + c128 FGMRES",
         "mixed_bf16": "c64 sweeps (3xBF16 tensor-core substitutions) + c128 FGMRES",
         "mixed_fp32": "c64 sweeps (FP32 CUDA-core substitutions) + c128 FGMRES"}
SPLIT_KIND = {"mixed": "tf32", "mixed_bf16": "bf16", "mixed_fp32": "fp32"}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the substitution and
# trace kernels, from one ncu capture of each kernel as it stands, on the same workload and launch
# shape (panel width, panels per CTA; cold, serialised replay: written data that stays in L2 is
# not counted).  The substitution figure is the mean over the launches of one solve (the first
# own-source launch skips most local problems as zero).  HBM_TRAFFIC: the same counters per DDM
# application for the assembly and extraction families.
SUBST_TRAFFIC = {("mixed", "layer2d_1024", 16, 2): 9808.2e6 / 4}
TRACE_TRAFFIC = {("mixed", "const2d_640"): 40.26e6 + 0.08e6}
TRACE_TC_TRAFFIC = {("mixed", "layer2d_1024"): 1030.9e6 + 822.7e6}
HBM_TRAFFIC = {("mixed", "layer2d_1024"): {"assemble": 11619.9e6 / 2, "extract": 4621.4e6 / 2}}


def roofline_entry(stats, work, ddm_apps, args, geometry=None, mma_rate=None):
    """Rooflines of the two sweep kernel families from their event-timed totals.

    work = (substitution flops, trace-map flops) of one DDM application (dds_work_per_ddm:
    16 Ml Mb^2 flop per local solve; 8 x routed map rows x received inputs per sweep, subdomain
    and RHS); ddm_apps = DDM applications in the profiled solves.  Achieved = algorithmic flops /
    device time of the family.  Peaks: the tensor-core substitutions take the dense tensor rate of
    their piece type divided by the three split products each useful product costs (TF32 =
    measured BF16 rate x 1.1/2.25, the nominal TF32:BF16 ratio); FP32 CUDA-core kernels take
    152 SMs x 128 lanes x 2 flop x 2070 MHz.  The tensor peaks are the measured burst rate: each
    launch is timed alone, within solves of milliseconds.  The entry of the family with the larger
    device time is the line's roofline; all are listed.  mma_rate: the dense rate of the piece type
    measured on this GPU by dds_tensor_rate (TF/s of pieces); a tensor entry then also gives its
    fraction of that rate / 3 (`frac_of_mma_rate`).
    """
    peaks, src = _peaks()
    geo = geometry or {}
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    kind = SPLIT_KIND.get(args.precision, "fp32")
    entries = []

    def with_rate(e):
        if mma_rate and e.get("bound") == "tensor":
            e["mma_rate_peak"] = mma_rate / 3.0
            e["frac_of_mma_rate"] = e["achieved"] / (mma_rate / 3.0)
        return e

    n_s, ms_s = stats["subst"]
    if n_s > 0 and ms_s > 0 and work[0] > 0:
        achieved = work[0] * ddm_apps / (ms_s / 1e3) / 1e12
        if kind != "fp32":
            # the burst peak: each launch is timed alone, inside solves of milliseconds
            bf16 = peaks["bf16_tflops"]
            base = bf16 * (1.1 / 2.25) if kind == "tf32" else bf16
            peak = base / 3.0
            big = (geometry or {}).get("Mb", 0) > 128
            name = (f"k_big_mma<{kind}> + k_big_epi (stage-parallel block forward+back "
                    f"substitution of blocks wider than 128 nodes, 3x{kind.upper()} split "
                    f"products on tcgen05)" if big else
                    f"k_subst_tc<{kind}> (block forward+back substitution, 3x{kind.upper()} "
                    f"split products on tcgen05, two-sided chain)")
            e = {"kernel": name, "bound": "tensor",
                 "peak_source": f"{src} bf16 burst {bf16:.0f} TF/s"
                                + (" x 1.1/2.25 (nominal TF32:BF16)" if kind == "tf32" else "")
                                + " / 3 split products"}
        else:
            peak = fp32_peak
            e = {"kernel": "k_subst_stream<float> (block forward+back substitution)", "bound": "alu",
                 "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
        e.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                  "traffic": SUBST_TRAFFIC.get((args.precision, args.workload,
                                                geo.get("panel_width"), geo.get("panels_per_cta"))),
                  "launches": n_s, "avg_launch_ms": ms_s / n_s, "device_ms": ms_s})
        entries.append(with_rate(e))
    n_t, ms_t = stats["trace_step"]
    if n_t > 0 and ms_t > 0 and work[1] > 0:
        achieved = work[1] * ddm_apps / (ms_t / 1e3) / 1e12
        tc = (geometry or {}).get("trace_kernel", 1) == 0 and kind != "fp32"
        if tc:
            bf16 = peaks["bf16_tflops"]
            peak = (bf16 * (1.1 / 2.25) if kind == "tf32" else bf16) / 3.0
            e = {"kernel": f"k_trace_tc<{kind}> (every trace solve of a DDM application as "
                           f"3x{kind.upper()} split-product GEMMs on tcgen05, one cooperative "
                           f"launch)", "bound": "tensor",
                 "peak_source": f"{src} bf16 burst {bf16:.0f} TF/s"
                                + (" x 1.1/2.25 (nominal TF32:BF16)" if kind == "tf32" else "")
                                + " / 3 split products",
                 "traffic": TRACE_TC_TRAFFIC.get((args.precision, args.workload))}
        else:
            peak = fp32_peak
            e = {"kernel": "k_trace_sweeps<float> (every trace step of a DDM application, "
                           "one cooperative launch, FP32 CUDA cores)", "bound": "alu",
                 "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                 "traffic": TRACE_TRAFFIC.get((args.precision, args.workload))}
        e.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                  "frac": achieved / peak, "launches": n_t, "avg_launch_ms": ms_t / n_t,
                  "device_ms": ms_t})
        entries.append(with_rate(e))
    # HBM-side kernels of the trace plan, from their algorithmic bytes per DDM application:
    #   assembly (two launches): every local right-hand side written once, the source read once
    #   over the owned ranges (which tile the global grid), and the final launch reads the trace
    #   slots of every sweep;  extraction (two launches): the raw trace lines read and written,
    #   then the owned nodes read locally and written to the global field (FP64).
    if geo.get("plan") == 2 and geo.get("Nloc"):   # DDS_PLAN_TRACE
        hbm = peaks.get("hbm_gbs", 6800.0)
        el = 16 if args.precision == "fp64" else 8
        R, Ng, Nl, T = geo["nrhs"], geo["Nglob"], geo["Nloc"], geo["T"]
        cols = R * geo["nsub"]
        L = geo["sweeps"]
        fam = {
            "assemble": ("k_assemble (local right-hand sides: source + trace potentials)",
                         2 * cols * Nl * el + 2 * R * Ng * 16 + cols * L * T * el),
            "extract": ("k_extract (trace lines, owned nodes to the global field)",
                        2 * cols * T * el + R * Ng * (el + 16)),
        }
        measured = HBM_TRAFFIC.get((args.precision, args.workload), {})
        for key, (name, nbytes) in fam.items():
            n_k, ms_k = stats.get(key, (0, 0.0))
            if n_k > 0 and ms_k > 0:
                achieved = nbytes * ddm_apps / (ms_k / 1e3) / 1e9
                # per launch (two launches per DDM application), like the algorithmic bytes
                traffic = measured[key] / 2 if key in measured else None
                entries.append({"kernel": name, "bound": "hbm",
                                "peak_source": f"{src} hbm_gbs", "achieved": achieved,
                                "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                                "traffic": traffic, "bytes_per_launch": nbytes / 2,
                                "launches": n_k, "avg_launch_ms": ms_k / n_k, "device_ms": ms_k})
    if not entries:
        return None, []
    main = dict(max(entries, key=lambda e: e["device_ms"]))
    main["family_share"] = {k: v[1] for k, v in stats.items()}
    return main, entries


# Table 5 as printed: GMRES iterations and solve seconds of the trace-transfer method on the
# paper's cluster (N x N subdomains of 300^2, one core per subdomain)
TABLE5_PAPER = {2: (3, 29.3), 4: (3, 64.4), 8: (3, 123.5), 16: (3, 268.4), 32: (4, 715.3)}


def run_table5(args):
    """The weak-scaling series of Table 5: fixed 300^2 subdomains (30-point PML), N x N
    partitions at the printed frequencies, one right-hand side of four approximated delta
    sources (Eq. 5.4), FGMRES to 1e-6 with the DDM as preconditioner (one round)."""
    import torch

    from paper_2003_02585_gb300 import build as lbuild
    from paper_2003_02585_gb300 import dds, synth

    torch.cuda.set_device(0)
    lbuild.build()
    series = []
    for N in [int(x) for x in args.table5.split(",") if x]:
        wl = synth.workload(f"table5_{N}")
        t0 = time.perf_counter()
        ctx = dds.Context(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength,
                          precision=args.precision, plan=args.plan)
        setup_s = time.perf_counter() - t0
        f = torch.from_numpy(ctx.extend(wl.f)).cuda()
        ctx.solve(f, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)      # warm-up (graphs)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            u, it, rel = ctx.solve(f, tol=args.tol, maxit=args.maxit, rounds=wl.rounds)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        info = ctx.info()
        series.append({"parts": f"{N}x{N}", "grid": list(wl.n), "freq": wl.meta["paper_freq"],
                       "n_iter": it, "relres": float(max(rel)), "solve_ms": min(ms),
                       "setup_s": setup_s, "factors": info["n_factors"],
                       "factor_gb": info["factor_bytes"] / 1e9,
                       "paper_n_iter": TABLE5_PAPER[N][0], "paper_solve_s": TABLE5_PAPER[N][1]})
        ctx.close()
        del f
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "Table 5 weak scaling: FGMRES iterations and solve time, one RHS",
                      "unit": "ms", "higher_is_better": False, "precision": args.precision,
                      "data": "synthetic (Eq. 5.4 sources)", "series": series,
                      "paper_context": "trace transfer on the paper's cluster, one core per "
                                       "subdomain; other hardware"}), flush=True)
    return 0


def run_serving(args):
    """Serving workload: Poisson request stream (each request 1-32 point sources) over three
    cached media, continuous batching per medium; RHS/s and per-request p50/p99 latency."""
    import torch

    from paper_2003_02585_gb300 import build as lbuild
    from paper_2003_02585_gb300 import serving

    torch.cuda.set_device(0)
    lbuild.build()
    rng = np.random.default_rng(5)
    media = serving.serving_media()
    reqs = serving.poisson_requests(rng, args.serve_requests, args.serve_rate, len(media))
    out = serving.run(reqs, media, budget_bytes=args.serve_budget_gb * 1e9, tol=args.tol,
                      maxit=args.serve_maxit, rounds=args.rounds or 3)
    lat = np.sort(out["latency_s"]) * 1e3
    line = {
        "metric": METRIC, "value": out["rhs"] / out["wall_s"], "unit": "RHS/s", "n_gpus": 1,
        "steps": len(reqs), "warmup": 0, "ms_per_step": 1e3 * out["wall_s"] / len(reqs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 sweeps + c128 FGMRES", "data": "synthetic",
        "config": {"workload": "serving: Poisson requests (1-32 sources) over 256^2 constant, "
                               "512^2 two-layer and 1024^2 random media, continuous batching",
                   "requests": len(reqs), "arrival_rate_per_s": args.serve_rate,
                   "slots": out["slots"], "launch_shapes": out["launch_shapes"],
                   "budget_gb": args.serve_budget_gb,
                   "maxit": args.serve_maxit},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "setup_seconds": out["setup_s"], "max_relres": out["max_relres"],
        "server_steps": out["steps"], "max_iters_per_medium": out["max_iters"],
        "p99_ms_per_medium": [1e3 * v for v in out["p99_s"]],
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--maxit", type=int, default=40)
    ap.add_argument("--plan", default="auto", choices=["auto", "direct", "trace"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_bf16", "mixed_fp32"],
                    help="single-precision sweep variant of the timed solver")
    ap.add_argument("--table5", default="2,4,8,16",
                    help="partitions N of the Table 5 series (--workload table5)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of timing the candidates")
    ap.add_argument("--shape", default=None,
                    help="pin the launch shapes instead of autotuning: 'panel width,panels per "
                         "CTA,trace kernel' (trace kernel 0 = tensor cores, 1/2 = CUDA cores)")
    ap.add_argument("--variants", default="mixed_bf16,mixed_fp32",
                    help="other sweep variants timed the same way and reported beside the line")
    ap.add_argument("--rounds", type=int, default=None,
                    help="DDM rounds per preconditioner application (default: the workload's)")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed steps of the FP64 comparator (default: --steps)")
    ap.add_argument("--fp64-warmup", type=int, default=None,
                    help="warm-up solves of the FP64 comparator (default: --warmup; its solve to "
                         "1e-10 for the accuracy check precedes them)")
    ap.add_argument("--nrhs", type=int, default=None,
                    help="right-hand sides of the workload (default: its own count; smaller "
                         "counts make the small cases the profiler captures)")
    ap.add_argument("--also", default="const2d_640,table5_2,table5_4",
                    help="other workloads measured briefly and reported beside the headline "
                         "('none' for none)")
    ap.add_argument("--also-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-rate", type=float, default=10.0, help="requests per second")
    ap.add_argument("--serve-budget-gb", type=float, default=180.0)
    ap.add_argument("--serve-maxit", type=int, default=16,
                    help="FGMRES iterations a serving slot is sized for (slot memory grows with it)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "table5":
        return run_table5(args)
    if args.workload == "serve":
        return run_serving(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
