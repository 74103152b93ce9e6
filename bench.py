#!/usr/bin/env python
"""Benchmark: Helmholtz solves/s to relative residual 1e-6, MP-1, k = 100, n = 1025.

Workload (one "step" = one full solve of the hot path): MP-1 (Dirichlet),
point source 1/h^2 at (1/2, 1/2), k = 100, n = 1025 (h = 1/1024), 16 x 16
square subdomains with 2 node layers of overlap, SHS2 preconditioner with the
B_2 coarse space on H = 1/32, right-preconditioned GMRES without restart from
u = 0 to ||f - A u|| <= 1e-6 ||f||.  The headline precision is MIXED
(complex64 stencil, transfers and subdomain solves inside FP64 flexible GMRES,
FP64 coarse solve); the FP64 path is timed beside it.  The preconditioner is
set up once before the timed region (set-up time is reported separately).

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (bounded sample, extrapolated per solve).
"""
from __future__ import annotations

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

N, K_WAVE, NSUB, OVERLAP, P_COARSE, TOL, MAXIT = 1025, 100.0, 16, 2, 32, 1e-6, 1000
WORKLOAD = ("MP-1 Dirichlet, k=100, n=1025 (h=1/1024), centre point source, 16x16 subdomains, overlap 2, "
            "SHS2 with B2 coarse space H=1/32, GMRES (no restart) to rel. residual 1e-6")
METRIC = "Helmholtz solves/s to rel. residual 1e-6 (k=100,n=1025), FP64 vs mixed; HBM %"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-wide-arm", action="store_true",
                    help="skip the arm whose Krylov basis keeps complex64 remainders (about 48 bits)")
    ap.add_argument("--no-dedup-arm", action="store_true",
                    help="skip the MIXED arm with every subdomain factored separately")
    ap.add_argument("--stream", action="store_true",
                    help="issue the Arnoldi steps as stream launches (default: CUDA graphs of 8 steps, "
                         "HZS_SOLVE_GRAPH); the other issue mode is timed beside the value")
    ap.add_argument("--no-alt-arm", action="store_true",
                    help="skip the solves issued the other way (stream launches vs CUDA graphs)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="launch the subdomain solve with its default shape instead of the set-up autotuner's")
    ap.add_argument("--workload", choices=["headline", "batched"], default="headline",
                    help="batched: the MP-2 multi-problem batch (64 right-hand sides for each of "
                         "(k, n) = (25, 257), (50, 257), (100, 513)) instead of the headline solve")
    ap.add_argument("--nrhs", type=int, default=64, help="right-hand sides per problem (batched workload)")
    ap.add_argument("--cpu-steps", type=int, default=6, help="Arnoldi steps in the oracle sample")
    # smaller MP-1 instances of the same path, for profiling captures only
    ap.add_argument("--n", type=int, default=1025)
    ap.add_argument("--k", type=float, default=100.0)
    ap.add_argument("--nsub", type=int, default=16)
    ap.add_argument("--coarse-ratio", type=int, default=32)
    ap.add_argument("--maxit", type=int, default=1000)
    a = ap.parse_args()
    global N, K_WAVE, NSUB, P_COARSE, WORKLOAD, MAXIT
    MAXIT = a.maxit
    if (a.n, a.k, a.nsub, a.coarse_ratio) != (N, K_WAVE, NSUB, P_COARSE):
        N, K_WAVE, NSUB, P_COARSE = a.n, a.k, a.nsub, a.coarse_ratio
        WORKLOAD = (f"MP-1 Dirichlet, k={a.k:g}, n={a.n}, centre point source, {a.nsub}x{a.nsub} subdomains, "
                    f"overlap 2, SHS2 with B2 coarse space H={a.coarse_ratio}h, GMRES to rel. residual 1e-6 "
                    "(profiling instance, not the headline workload)")
    return a


# ----------------------------------------------------------------- distributed
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """Largest x over the ranks of the default process group (x itself for one rank)."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: int, ms_max: float, world: int) -> float:
    """Whole-job rate of N independent replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(rows[0][2]),
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


# ----------------------------------------------------------------- CPU oracle (baseline / reference arm)
def oracle_sample(steps: int, iterations: int):
    """Times the FP64 CPU oracle on this workload: set-up, then ``steps`` Arnoldi steps
    of its GMRES; the per-solve time at ``iterations`` steps is extrapolated from the
    measured preconditioner + operator cost per step and the measured cost of one
    Gram-Schmidt projection (the orthogonalisation grows linearly with the step)."""
    import numpy as np

    from oracle import DIRICHLET, B2, Problem, Schwarz, SHS2, gmres
    from paper_2408_03571_gb300.inputs import point_source

    t0 = time.perf_counter()
    prob = Problem(N, DIRICHLET, K_WAVE ** 2)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, NSUB, OVERLAP, SHS2, B2, P_COARSE)
    t_setup = time.perf_counter() - t0
    f = prob.grid_to_vec(point_source(N))
    # preconditioner + operator per step
    t0 = time.perf_counter()
    for _ in range(2):
        A @ M.apply(f)
    t_pm = (time.perf_counter() - t0) / 2
    # one modified Gram-Schmidt projection (inner product + update) on a vector
    v = f / np.linalg.norm(f)
    w = np.array(f)
    t0 = time.perf_counter()
    for _ in range(20):
        h = np.vdot(v, w)
        w = w - h * v
    t_proj = (time.perf_counter() - t0) / 20
    # a real run of the oracle's GMRES for a few steps (checks the model)
    t0 = time.perf_counter()
    res = gmres(lambda x: A @ x, M.apply, f, TOL, steps)
    t_run = time.perf_counter() - t0
    model_run = steps * t_pm + t_proj * steps * (steps + 1) / 2
    it = iterations
    t_solve = it * t_pm + t_proj * it * (it + 1) / 2
    return {
        "t_setup_s": t_setup, "t_precond_plus_operator_s": t_pm, "t_projection_s": t_proj,
        "t_sample_run_s": t_run, "sample_model_s": model_run, "iterations_assumed": it,
        "t_solve_extrapolated_s": t_solve, "sample_steps": res.iterations,
    }


def basis_dtype(bits: int) -> str:
    return {32: "f32 + bf16 remainder pairs (~32 bits)", 48: "double-float (2 x f32) pairs (~48 bits)",
            53: "c128"}.get(bits, f"{bits}-bit")


def cpu_cores_used():
    # numpy's vector ops used here are single-threaded; SuperLU is single-threaded
    return 1


def reference_arm(args, world, rank):
    if rank != 0:
        return
    iters_assumed = 372   # the mixed GPU solve's iteration count at this workload (measured)
    vals = []
    for _ in range(args.warmup):
        pass   # the oracle has no warm-up effects worth paying minutes for
    last = None
    for _ in range(max(1, args.steps)):
        last = oracle_sample(args.cpu_steps, iters_assumed)
        vals.append(1.0 / last["t_solve_extrapolated_s"])
    v = statistics.median(vals)
    sample = (f"oracle (numpy/scipy FP64) at the full workload: set-up, then {args.cpu_steps} GMRES steps; "
              f"per-solve time extrapolated to {iters_assumed} steps from the measured per-step "
              f"preconditioner+operator time and per-projection Gram-Schmidt time")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cpu_cores_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "detail": last}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm
# (k, n, subdomains per axis) of the batched MP-2 workload: 64-node subdomains, B_2 with
# H = 32h; (200, 1025) of the same family does not converge (kH = 6.25) and is left out
BATCHED = ((25.0, 257, 4), (50.0, 257, 4), (100.0, 513, 8))


def batched_arm(args, world, rank, local):
    """All problems of the batch solved concurrently (hzs_solve_batched), every right-hand
    side a point source at a seeded interior node; one step = the whole batch."""
    import numpy as np
    import torch

    from paper_2408_03571_gb300 import build, hzs
    from paper_2408_03571_gb300.inputs import point_source, random_source_nodes

    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    hzs.load()
    dev = torch.device("cuda", local)
    grids, precs, rhs_host, rhs = [], [], [], []
    t0 = time.perf_counter()
    for i, (k, n, nsub) in enumerate(BATCHED):
        # a stream per problem, so that the problems' kernels overlap on the GPU
        g = hzs.Grid(n, hzs.SOMMERFELD, k=k, nsub=nsub, overlap=2, stream=torch.cuda.Stream(dev))
        grids.append(g)
        precs.append(hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 32, hzs.MIXED,
                                        autotune=0 if args.no_autotune else 1))
        nodes = random_source_nodes(n, args.nrhs, 1000 + i)
        fh = torch.from_numpy(np.stack([point_source(n, nd) for nd in nodes])).pin_memory()
        rhs_host.append(fh)
        rhs.append(fh.to(dev))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        hzs.solve_batched(precs, rhs, TOL, MAXIT, graph=args.graph)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = None
    for _ in range(args.steps):
        _, infos = hzs.solve_batched(precs, rhs, TOL, MAXIT, graph=args.graph)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    # end to end: right-hand sides from pinned host memory, solutions back, inside the timed region
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        fd = [f.to(dev, non_blocking=True) for f in rhs_host]
        stream.synchronize()            # the copies ran on this stream; the solves run on the problems'
        outs, _ = hzs.solve_batched(precs, fd, TOL, MAXIT, graph=args.graph)
        for u in outs:
            u.cpu()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1), world, dev)
    nsol = sum(len(r) for r in infos)
    shapes = [P.info() for P in precs]
    per = []
    for (k, n, nsub), res, sh in zip(BATCHED, infos, shapes):
        its = [r.iterations for r in res]
        per.append({"k": k, "n": n, "nrhs": len(res), "iterations_max": max(its),
                    "subdomain_solve_shape": {key: sh[key] for key in ("tile_group", "tile_stages",
                                                                       "tile_threads_per_row", "autotuned",
                                                                       "apply_us_default", "apply_us_tuned")},
                    "iterations_mean": float(np.mean(its)),
                    "converged": int(sum(r.converged for r in res)),
                    "relres_true_max": max(r.relres_true for r in res)})
    for P in precs:
        P.close()
    for g in grids:
        g.close()
    if rank != 0:
        return
    bytes_io = sum(f.numel() * 16 for f in rhs_host)
    line = {
        "metric": "batched MP-2 Helmholtz solves/s to rel. residual 1e-6 (3 problems x %d right-hand sides)"
                  % args.nrhs,
        "value": replica_throughput(nsol, ms / args.steps, world), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 preconditioner; Arnoldi basis as " + basis_dtype(min(r.basis_bits for res in infos for r in res))
                 + "; f64 Hessenberg",
        "data": "synthetic",
        "config": {"workload": "MP-2 batch: (k, n) = (25, 257), (50, 257), (100, 513), 64-node subdomains, "
                               "overlap 2, SHS2 with B2 H=32h, point sources at seeded nodes, all problems "
                               "solved concurrently, right-hand sides of a problem in lockstep",
                   "issue": "CUDA graphs of 8 Arnoldi steps" if args.graph else "stream launches",
                   "l2": "working set larger than L2; no flush needed", "parallelism": f"replicas x{world}"},
        "problems": per, "setup_s": setup_s,
        "e2e": {"value": replica_throughput(nsol, ms_e2e / args.steps, world), "unit": "solves/s",
                "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io},
    }
    print(json.dumps(line), flush=True)


def gpu_arm(args, world, rank, local):
    import torch

    from paper_2408_03571_gb300 import build, hzs
    from paper_2408_03571_gb300.inputs import point_source

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    hzs.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    f_host = torch.from_numpy(point_source(N)).pin_memory()
    f = f_host.to(dev)
    grid = hzs.Grid(N, hzs.DIRICHLET, k=K_WAVE, nsub=NSUB, overlap=OVERLAP)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    def timed_solves(P, steps, warmup, e2e=False, profile=False, wide=False, graph=False):
        u = torch.empty_like(f)
        u_host = torch.empty_like(f_host).pin_memory()
        infos = []
        for _ in range(warmup):
            P.solve(f, TOL, MAXIT, out=u, wide_basis=wide, graph=graph)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            if e2e:
                fd = f_host.to(dev, non_blocking=True)
                _, inf = P.solve(fd, TOL, MAXIT, out=u, profile=profile, wide_basis=wide, graph=graph)
                u_host.copy_(u, non_blocking=True)
            else:
                _, inf = P.solve(f, TOL, MAXIT, out=u, profile=profile, wide_basis=wide, graph=graph)
            infos.append(inf[0])
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        return max_over_ranks(ms, world, dev), infos, u

    out = {}
    # ---- mixed (headline)
    t0 = time.perf_counter()
    Pm = hzs.Preconditioner(grid, hzs.SHS2, hzs.COARSE_B2, P_COARSE, hzs.MIXED,
                            autotune=0 if args.no_autotune else 1)
    torch.cuda.synchronize()
    setup_mixed_s = time.perf_counter() - t0
    shape = Pm.info()
    # the headline value: solves without per-launch events
    clk = ClockSampler(local)
    clk.start()
    ms_tot, infos_plain, u = timed_solves(Pm, args.steps, args.warmup, graph=args.graph)
    clocks = clk.stop()
    # the same solves with CUDA events around every launch: phase times and the roofline
    ms_prof, infos, _ = timed_solves(Pm, args.steps, 0, profile=True)
    # the other way of issuing the Arnoldi steps (stream launches, or graphs with --stream)
    issue_alt = None
    if not args.no_alt_arm:
        ms_alt, infos_alt, _ = timed_solves(Pm, args.steps, 1, graph=not args.graph)
        issue_alt = {"value": replica_throughput(args.steps, ms_alt, world), "unit": "solves/s",
                     "ms_per_step": ms_alt / args.steps, "iterations": infos_alt[-1].iterations,
                     "relres_true": infos_alt[-1].relres_true,
                     "issue": "stream launches" if args.graph else "CUDA graphs of 8 Arnoldi steps"}
    ms_e2e, infos_e2e, _ = timed_solves(Pm, args.steps, 0, e2e=True, graph=args.graph)
    # ---- the same solve with the basis remainders kept as complex64 (about 48 bits)
    wide = None
    if not args.no_wide_arm:
        ms_w, infos_w, _ = timed_solves(Pm, max(1, args.steps // 2), 1, profile=True, wide=True)
        i0 = infos_w[-1]
        wide = {"value": replica_throughput(len(infos_w), ms_w, world), "unit": "solves/s",
                "ms_per_step": ms_w / len(infos_w), "iterations": i0.iterations,
                "relres_est": i0.relres_est, "relres_true": i0.relres_true, "basis_bits": i0.basis_bits,
                "t_orth_ms": i0.t_orth_ms,
                "note": "Krylov basis as complex64 + complex64 remainder (16 B an entry; the default "
                        "for tol < 1e-7)"}
    Pm.close()
    # ---- MIXED with one factor per subdomain (no sharing of identical factors): the
    # subdomain solves then stream 256 distinct factor sets per apply, as for a kappa field
    dedup_off = None
    if not args.no_dedup_arm:
        Pn = hzs.Preconditioner(grid, hzs.SHS2, hzs.COARSE_B2, P_COARSE, hzs.MIXED, dedup_tiles=False)
        ms_n, infos_n, _ = timed_solves(Pn, max(1, args.steps // 2), 1, profile=True)
        Pn.close()
        i0 = infos_n[-1]
        dedup_off = {"value": replica_throughput(len(infos_n), ms_n, world), "unit": "solves/s",
                     "ms_per_step": ms_n / len(infos_n), "iterations": i0.iterations,
                     "relres_true": i0.relres_true, "t_precond_ms": i0.t_precond_ms,
                     "note": "every subdomain factor stored and streamed separately (no sharing of "
                             "identical factors)"}
    # ---- FP64 arm
    fp64 = None
    if not args.no_fp64:
        t0 = time.perf_counter()
        Pd = hzs.Preconditioner(grid, hzs.SHS2, hzs.COARSE_B2, P_COARSE, hzs.FP64)
        torch.cuda.synchronize()
        setup_fp64_s = time.perf_counter() - t0
        ms_d, infos_d, _ = timed_solves(Pd, max(1, args.steps // 2), 1, profile=True)
        Pd.close()
        i0 = infos_d[-1]
        fp64 = {"value": replica_throughput(len(infos_d), ms_d, world), "unit": "solves/s",
                "ms_per_step": ms_d / len(infos_d), "iterations": i0.iterations,
                "relres_true": i0.relres_true, "setup_s": setup_fp64_s,
                "t_precond_ms": i0.t_precond_ms, "t_matvec_ms": i0.t_matvec_ms, "t_orth_ms": i0.t_orth_ms}
    grid.close()

    # ---- roofline of the dominant kernels: the two passes of the delayed CGS2 over
    # the double-float basis, complex64 leading words + remainders: eb = 12 B per basis
    # entry with bf16 remainders (tol >= 1e-7), 16 B with complex64 remainders.
    # Algorithmic HBM bytes at step j (Nu unknowns):
    #   dot pass    k_dcgs_dot:    leading words of basis vectors 0..j-1, u~_j and w (8 (j + 2) Nu)
    #   update pass k_dcgs_update: basis vectors 0..j-1 (eb j Nu), u~_j and w read and written (4 eb Nu)
    # Step j = it completes the last column (dot pass only); its update returns at once.
    last = infos[-1]
    it = last.iterations
    Nu = (N - 2) ** 2
    eb = 12 if last.basis_bits == 32 else 16
    dot_bytes = sum(8 * (j + 2) * Nu for j in range(it + 1))
    upd_bytes = sum(eb * (j + 4) * Nu for j in range(it))
    t_dot = statistics.mean(i.t_orth_dot_ms for i in infos) * 1e-3
    t_upd = statistics.mean(i.t_orth_update_ms for i in infos) * 1e-3
    orth_s = statistics.mean(i.t_orth_ms for i in infos) * 1e-3
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = ("MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)" if "hbm_gbs" in peaks
                else "fallback 6800 GB/s")

    def pass_roofline(name, nbytes, t):
        a = nbytes / t / 1e9 if t > 0 else 0.0
        return {"kernel": name, "bound": "hbm", "achieved": a, "peak": hbm_peak, "unit": "GB/s",
                "frac": a / hbm_peak, "traffic": None, "peak_source": peak_src,
                "bytes_per_solve": nbytes, "time_per_solve_s": t,
                "timing": "CUDA events around every launch of the kernel on the solve stream, over a "
                          "timed region of the same number of solves as the value's"}
    r_dot = pass_roofline("k_dcgs_dot (delayed CGS2 multi-dot on the leading words of the basis)", dot_bytes,
                          t_dot)
    r_upd = pass_roofline("k_dcgs_update (delayed CGS2 basis update, double-float)", upd_bytes, t_upd)
    # DRAM traffic of the two passes from one ncu capture per basis width (MP-1 k=100
    # n=513, the launches of step 200), as a ratio to the algorithmic bytes of that
    # launch; traffic grows with the units processed, so the average launch here is
    # scaled by those ratios.  None: no capture of the current kernel.
    dot_ratio = (1.021, "430.9 MB against 421.9 MB")
    traffic_ratio = {16: {"dot": dot_ratio, "upd": None},
                     12: {"dot": dot_ratio, "upd": (1.079, "689.7 MB against 639.2 MB")}}[eb]
    for r_, nbytes, nl, key in ((r_dot, dot_bytes, it + 1, "dot"), (r_upd, upd_bytes, it, "upd")):
        r_["launches"] = nl
        r_["bytes_per_launch"] = nbytes / nl
        r_["basis_bytes_per_entry"] = 8 if key == "dot" else eb
        tr = traffic_ratio[key]
        r_["traffic"] = None if tr is None else tr[0] * nbytes / nl
        r_["traffic_source"] = (
            "no ncu capture of this kernel version" if tr is None else
            "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch (n=513, step 200: "
            f"{tr[1]} algorithmic = {tr[0]}), scaled to this workload's average launch")
    roofline = dict(r_upd if t_upd >= t_dot else r_dot)
    roofline["other_pass"] = r_dot if t_upd >= t_dot else r_upd
    roofline["orth_group"] = {"time_per_solve_s": orth_s,
                              "achieved_gbs": (dot_bytes + upd_bytes) / orth_s / 1e9,
                              "note": "both passes plus the reduction, Givens and scale kernels"}
    if fp64 is not None:
        # all-FP64 CGS2: 4 passes x (j+1) Nu complex multiply-adds (8 flops each) on the FP64 pipe
        fp64_peak = 2.0 * 2.0 * 152 * 2.070e9     # 2 DFMA/clk/SM x 2 flops x 152 SMs x 2070 MHz
        it64 = fp64["iterations"]
        flops64 = sum(32.0 * (j + 1) * Nu for j in range(it64))
        t64 = fp64["t_orth_ms"] * 1e-3
        fp64["roofline"] = {"kernel": "CGS2 orthogonalisation, FP64 (k_multidot<double2> + k_axpy_multi)",
                            "bound": "alu", "achieved": flops64 / t64 / 1e12, "peak": fp64_peak / 1e12,
                            "unit": "TFLOP/s", "frac": flops64 / t64 / fp64_peak,
                            "peak_source": "FP64 pipe: 2 DFMA/clk/SM x 152 SMs x 2070 MHz"}

    value = replica_throughput(args.steps, ms_tot, world)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 preconditioner; Arnoldi basis as " + basis_dtype(last.basis_bits) + "; f64 Hessenberg, "
                 "coarse solve, outer operator and solution",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "mixed", "n": N, "k": K_WAVE, "nsub": NSUB,
                   "overlap": OVERLAP, "coarse_ratio": P_COARSE, "tol": TOL, "basis_bits": last.basis_bits,
                   "l2": "working set larger than L2 (Krylov basis ~6 GB); no flush needed",
                   "issue": "CUDA graphs of 8 Arnoldi steps" if args.graph else "stream launches",
                   "parallelism": f"replicas x{world}"},
        "iterations": infos_plain[-1].iterations, "relres_est": infos_plain[-1].relres_est,
        "relres_true": infos_plain[-1].relres_true,
        "setup_s": setup_mixed_s,
        "subdomain_solve_shape": shape,
        "profiled": {"value": replica_throughput(args.steps, ms_prof, world), "unit": "solves/s",
                     "note": "the same solves with CUDA events around every launch (phases and roofline)"},
        "issue_alt": issue_alt,
        "phases_ms": {"precond": last.t_precond_ms, "matvec": last.t_matvec_ms, "orth": last.t_orth_ms,
                      "solve": last.t_solve_ms},
        "roofline": roofline,
        "e2e": {"value": replica_throughput(args.steps, ms_e2e, world), "unit": "solves/s",
                "h2d_bytes_per_step": N * N * 16, "d2h_bytes_per_step": N * N * 16},
        "gpu_launches": int(sum(i.launches for i in infos_plain)),
        "clocks": clocks,
        "fp64": fp64,
        "wide_basis": wide,
        "dedup_off": dedup_off,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = oracle_sample(args.cpu_steps, it)
        line["cpu_baseline"] = {
            "value": 1.0 / s["t_solve_extrapolated_s"], "unit": "solves/s", "cores": cpu_cores_used(),
            "kind": "oracle",
            "sample": (f"oracle set-up + {args.cpu_steps} GMRES steps at the full workload; per-solve time "
                       f"extrapolated to {it} steps ({s['t_solve_extrapolated_s']:.0f} s)"),
            "detail": s}
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    args.graph = not args.stream
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    if args.workload == "batched":
        batched_arm(args, world, rank, local)
        return
    gpu_arm(args, world, rank, local)


if __name__ == "__main__":
    main()
