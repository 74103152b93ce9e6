#!/usr/bin/env python
"""Benchmark: Helmholtz solves/s to relative residual 1e-6, MP-1, k = 100, n = 1025.

Workload (one "step" = one full solve of the hot path): MP-1 (Dirichlet),
point source 1/h^2 at (1/2, 1/2), k = 100, n = 1025 (h = 1/1024), 16 x 16
square subdomains with 2 node layers of overlap, SHS2 preconditioner with the
B_2 coarse space on H = 1/32, right-preconditioned flexible GMRES without
restart from u = 0 to ||f - A u|| <= 1e-6 ||f||.  The headline precision is
MIXED: complex64 stencil, transfers and subdomain solves, FP64 coarse solve,
and an FP64 Arnoldi process (FP64 basis, FP64-accurate reorthogonalisation and
update, FP64 Hessenberg least squares).  The preconditioner is set up once
before the timed region (set-up time is reported separately).  Beside the
headline: the FP64 path, the other orthogonalisations, and the other
configurations of the workload family (the small MP-1 case, MP-2 at n = 513,
the batched MP-2 set, the differentiable MP-2 solve), one solve each.

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (bounded sample per step, extrapolated per solve).
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
    ap.add_argument("--no-alt-orth", action="store_true",
                    help="skip the arms with the other orthogonalisations (all-FP64-FMA delayed CGS2, "
                         "double-float bases of 32 and 48 bits)")
    ap.add_argument("--no-dedup-arm", action="store_true",
                    help="skip the MIXED arm with every subdomain factored separately")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other configurations (small MP-1, MP-2 n=513, batched MP-2, gradient)")
    ap.add_argument("--stream", action="store_true",
                    help="issue the Arnoldi steps as stream launches (default: CUDA graphs of 8 steps, "
                         "HZS_SOLVE_GRAPH); the other issue mode is timed beside the value")
    ap.add_argument("--no-alt-arm", action="store_true",
                    help="skip the solves issued the other way (stream launches vs CUDA graphs)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="launch the subdomain solve with its default shape instead of the set-up autotuner's")
    ap.add_argument("--workload", choices=["headline", "batched"], default="headline",
                    help="batched: print the line of the batched MP-2 set (64 right-hand sides for each "
                         "(k, n)) instead of the headline solve")
    ap.add_argument("--nrhs", type=int, default=64, help="right-hand sides per problem (batched workload)")
    ap.add_argument("--cpu-steps", type=int, default=6, help="Arnoldi steps in an oracle sample (reference arm)")
    ap.add_argument("--oracle-full-solve", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--profile-solve", action="store_true",
                    help="set up, then run exactly one stream-issued MIXED solve of the workload and exit "
                         "(for profiler captures; prints its step count); with --workload batched: one "
                         "MP-2 problem (--k --n --nsub --coarse-ratio) with --nrhs point sources, solved once "
                         "untimed and once between cudaProfilerStart and cudaProfilerStop")
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
def _oracle_setup():
    from oracle import DIRICHLET, B2, Problem, Schwarz, SHS2
    from paper_2408_03571_gb300.inputs import point_source

    t0 = time.perf_counter()
    prob = Problem(N, DIRICHLET, K_WAVE ** 2)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, NSUB, OVERLAP, SHS2, B2, P_COARSE)
    f = prob.grid_to_vec(point_source(N))
    return prob, A, M, f, time.perf_counter() - t0


def oracle_full_solve():
    """One complete solve of the headline workload by the FP64 CPU oracle as it stands
    (right-preconditioned GMRES with modified Gram-Schmidt, SuperLU local solves), on
    one core; prints its timings as a JSON line (run as a child process)."""
    from oracle import gmres

    prob, A, M, f, t_setup = _oracle_setup()
    t0 = time.perf_counter()
    res = gmres(lambda x: A @ x, M.apply, f, TOL, MAXIT)
    t_solve = time.perf_counter() - t0
    print(json.dumps({"t_setup_s": t_setup, "t_solve_s": t_solve, "iterations": res.iterations,
                      "relres_true": res.relres_true, "converged": bool(res.converged)}), flush=True)


def start_oracle_child():
    """Starts oracle_full_solve in a fresh interpreter (before any CUDA call of this
    process), pinned to one thread of every numerical library."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    size = ["--n", str(N), "--k", str(K_WAVE), "--nsub", str(NSUB), "--coarse-ratio", str(P_COARSE),
            "--maxit", str(MAXIT)]
    return subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-full-solve", *size],
                            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)


def finish_oracle_child(proc, timeout_s: float):
    try:
        out, err = proc.communicate(timeout=timeout_s)
    except subprocess.TimeoutExpired:
        proc.kill()
        proc.communicate()
        return None, f"oracle solve did not finish within {timeout_s:.0f} s"
    for line in reversed(out.splitlines()):
        if line.startswith("{"):
            return json.loads(line), None
    return None, "oracle solve failed: " + err.strip().splitlines()[-1] if err.strip() else "no output"


def oracle_sample(prob, A, M, f, steps: int, iterations: int):
    """A bounded sample of the oracle on the full workload: ``steps`` Arnoldi steps of its
    GMRES (set-up done before), plus the measured cost of the preconditioner and operator
    and of one Gram-Schmidt projection on basis vectors that are not cache-resident.  The
    per-solve time at ``iterations`` steps is modelled from those two costs (the
    orthogonalisation grows linearly with the step): it * t_pm + t_proj * it (it + 1) / 2.
    The model is checked against one complete oracle solve of this workload (the GPU
    arm's cpu_baseline: 355 steps in 232 s measured, 236 s modelled); the sample run's
    own time is reported beside it."""
    import numpy as np

    from oracle import gmres

    t0 = time.perf_counter()
    A @ M.apply(f)
    t_pm = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    basis = [rng.standard_normal(f.shape[0]) + 1j * rng.standard_normal(f.shape[0]) for _ in range(24)]
    w = np.array(f)
    t0 = time.perf_counter()
    for v in basis:
        h = np.vdot(v, w)
        w = w - h * v
    t_proj = (time.perf_counter() - t0) / len(basis)
    t0 = time.perf_counter()
    res = gmres(lambda x: A @ x, M.apply, f, TOL, steps)
    t_run = time.perf_counter() - t0
    model = lambda it: it * t_pm + t_proj * it * (it + 1) / 2
    return {"t_precond_plus_operator_s": t_pm, "t_projection_s": t_proj, "t_sample_run_s": t_run,
            "sample_steps": res.iterations, "sample_modelled_s": model(res.iterations),
            "iterations_assumed": iterations, "t_solve_extrapolated_s": model(iterations)}


def basis_dtype(bits: int, kind: int) -> str:
    if kind in (1, 3):
        return "f64 (53 bits; stored as f32 head + 29-bit tail)" if kind == 1 else "c128"
    return {32: "f32 + bf16 remainder pairs (~32 bits)", 48: "double-float (2 x f32) pairs (~48 bits)",
            53: "c128"}.get(bits, f"{bits}-bit")


def reference_arm(args, world, rank):
    """The oracle on this machine's host cores, one bounded sample per step (the same metric,
    unit and workload as the GPU arm; there is no installable reference implementation)."""
    if rank != 0:
        return
    # one core, as stated in the line (the numerical libraries are loaded after this)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    iters_assumed = 355   # the oracle's own step count for this workload (its full solve, measured)
    prob, A, M, f, t_setup = _oracle_setup()
    for _ in range(min(args.warmup, 1)):
        A @ M.apply(f)
    samples, walls = [], []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        samples.append(oracle_sample(prob, A, M, f, args.cpu_steps, iters_assumed))
        walls.append(time.perf_counter() - t0)
    v = statistics.median(1.0 / s["t_solve_extrapolated_s"] for s in samples)
    sample = (f"per step: {args.cpu_steps} GMRES steps of the FP64 oracle (numpy/scipy, one core) at the full "
              f"workload plus its measured per-step preconditioner+operator and per-projection costs; "
              f"value = one solve of the oracle's {iters_assumed} steps modelled from them (set-up {t_setup:.1f} s, "
              f"once; the model is within 2 % of a complete oracle solve timed on the same host)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "detail": samples[-1]}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm
# Batched MP-2 set: (k, n, subdomains per axis, H/h).  For each k the smallest n of
# {257, 513, 1025} with kh <= 0.2, 64-node subdomains, and H the largest power-of-two
# multiple of h with kH <= 1 (the robustness condition of Section 5): kH = 0.78.
BATCHED = ((25.0, 257, 4, 8), (50.0, 257, 4, 4), (100.0, 513, 8, 4), (200.0, 1025, 16, 4))
# iteration cap of the batched set: 100, the cap of the paper's first two tables (Section 5);
# the set converges in at most 33 steps, and the Krylov spaces are sized by the cap
MAXIT_BATCHED = 100
# DRAM bytes (read + write) of one launch of each basis pass over its algorithmic bytes,
# from one ncu capture of the current kernels at the headline size (step j = 200)
TRAFFIC_RATIO = {"dot": 3736.3 / 3382.4, "update": 3525.2 / 3415.9}


def _peaks_file():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _ev_time(stream, fn, n):
    """Calls fn() n times between CUDA events on stream; returns (ms, last result)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = None
    for _ in range(n):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def _res(r):
    return {"iterations": r.iterations, "converged": bool(r.converged), "relres_true": r.relres_true}


def batched_set(args, dev, graph: bool):
    """All problems of the batched MP-2 set solved concurrently (hzs_solve_batched, every
    right-hand side a point source at a seeded node, each problem on its own stream);
    one step = the whole set.  Returns the measurements and the end-to-end timing."""
    import numpy as np
    import torch

    from paper_2408_03571_gb300 import hzs
    from paper_2408_03571_gb300.inputs import point_source, random_source_nodes

    grids, precs, rhs_host, rhs = [], [], [], []
    t0 = time.perf_counter()
    for i, (k, n, nsub, p) in enumerate(BATCHED):
        g = hzs.Grid(n, hzs.SOMMERFELD, k=k, nsub=nsub, overlap=2, stream=torch.cuda.Stream(dev))
        grids.append(g)
        precs.append(hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, hzs.MIXED,
                                        autotune=0 if args.no_autotune else 1))
        nodes = random_source_nodes(n, args.nrhs, 1000 + i)
        fh = torch.from_numpy(np.stack([point_source(n, nd) for nd in nodes])).pin_memory()
        rhs_host.append(fh)
        rhs.append(fh.to(dev))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    solve = lambda fs: hzs.solve_batched(precs, fs, TOL, MAXIT_BATCHED, graph=graph)
    solve(rhs)
    ms, (_, infos) = _ev_time(stream, lambda: solve(rhs), 1)

    def e2e():
        fd = [f.to(dev, non_blocking=True) for f in rhs_host]
        stream.synchronize()            # the copies ran on this stream; the solves run on the problems'
        outs, _ = solve(fd)
        return [u.cpu() for u in outs]
    ms_e2e, _ = _ev_time(stream, e2e, 1)
    per = []
    for (k, n, nsub, p), res, P in zip(BATCHED, infos, precs):
        its = [r.iterations for r in res]
        info = P.info()
        per.append({"k": k, "n": n, "nsub": nsub, "H_over_h": p, "kH": k * p / (n - 1), "nrhs": len(res),
                    "coarse_unknowns": info["coarse_unknowns"], "coarse_solver": info["coarse_solver"],
                    "iterations_max": max(its), "iterations_mean": float(np.mean(its)),
                    "converged": int(sum(r.converged for r in res)),
                    "relres_true_max": max(r.relres_true for r in res)})
    for P in precs:
        P.close()
    for g in grids:
        g.close()
    nsol = sum(len(r) for r in infos)
    return {"solves": nsol, "ms": ms, "ms_e2e": ms_e2e, "setup_s": setup_s, "problems": per,
            "bytes_io": sum(f.numel() * 16 for f in rhs_host)}


def other_configs(args, dev):
    """The other configurations of the workload family, each solved after one warm-up
    solve on its own handle: solves/s, steps and the FP64 true residual."""
    import torch

    from paper_2408_03571_gb300 import hzs
    from paper_2408_03571_gb300.inputs import distinct_interior_nodes, kappa_field, point_source

    stream = torch.cuda.current_stream(dev)
    out = {}

    def run(n, bc, k, nsub, p, kind, coarse, prec, tol, reps, kappa=None):
        g = hzs.Grid(n, bc, k=k, kappa=kappa, nsub=nsub, overlap=2)
        P = hzs.Preconditioner(g, kind, coarse, p, prec)
        f = torch.from_numpy(point_source(n)).to(dev)
        P.solve(f, tol, MAXIT, graph=args.graph)
        ms, (_, inf) = _ev_time(stream, lambda: P.solve(f, tol, MAXIT, graph=args.graph), reps)
        P.close()
        g.close()
        return dict(_res(inf[0]), value=reps / (ms * 1e-3), unit="solves/s", ms_per_solve=ms / reps)

    # small MP-1: n = 65, k = 20, 4 x 4 subdomains, B2 with H = 1/8, tol 1e-7
    out["mp1_n65_k20"] = {
        name: run(65, hzs.DIRICHLET, 20.0, 4, 8, hzs.SHS2, hzs.COARSE_B2, prec, 1e-7, 20)
        for name, prec in (("fp64", hzs.FP64), ("mixed", hzs.MIXED))}
    # MP-2: n = 513, k = 50, 8 x 8 subdomains, H = 1/16; one-level AS vs P1 vs B2, FP64 vs mixed
    cfg2 = {}
    for cname, kind, coarse in (("as1", hzs.AS1, hzs.COARSE_NONE), ("shs2_p1", hzs.SHS2, hzs.COARSE_P1),
                                ("shs2_b2", hzs.SHS2, hzs.COARSE_B2)):
        for pname, prec in (("fp64", hzs.FP64), ("mixed", hzs.MIXED)):
            cfg2[f"{cname}_{pname}"] = run(513, hzs.SOMMERFELD, 50.0, 8, 32, kind, coarse, prec, 1e-7, 2)
    out["mp2_n513_k50"] = cfg2
    # differentiable MP-2: n = 1025, kappa = (100 (1 + 0.2 g))^2, forward solve, adjoint solve of
    # the receivers' misfit and the kappa gradient, MIXED, tol 1e-6
    n = 1025
    kap = torch.from_numpy(kappa_field(n, 100.0, seed=2001)).to(dev)
    g = hzs.Grid(n, hzs.SOMMERFELD, kappa=kap, nsub=16, overlap=2)
    t0 = time.perf_counter()
    P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 32, hzs.MIXED, dedup_tiles=False)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    f = torch.from_numpy(point_source(n)).to(dev)
    rec = distinct_interior_nodes(n, 64, seed=2003)
    idx = torch.tensor([j * n + i for (i, j) in rec], device=dev)

    def fwd_adj():
        u, i1 = P.solve(f, TOL, MAXIT, graph=args.graph)
        r = torch.zeros_like(u).view(-1)
        r[idx] = u.view(-1)[idx]
        lam, i2 = P.adjoint_solve(r.view(n, n), TOL, MAXIT, graph=args.graph)
        P.kappa_gradient(u, lam)
        return i1[0], i2[0]
    fwd_adj()
    ms, (i1, i2) = _ev_time(stream, fwd_adj, 1)
    P.close()
    g.close()
    out["mp2_n1025_kappa_field_gradient"] = {
        "value": 1.0 / (ms * 1e-3), "unit": "forward+adjoint solve pairs/s", "ms_per_pair": ms, "setup_s": setup_s,
        "forward": _res(i1), "adjoint": _res(i2),
        "note": "forward solve, adjoint solve of the 64 receivers' values and the kappa gradient kernel"}
    return out


def gpu_arm(args, world, rank, local):
    # the oracle's full solve runs on one host core beside the GPU work (started before CUDA)
    child = start_oracle_child() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
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
    pipes = hzs.pipe_peaks()
    f_host = torch.from_numpy(point_source(N)).pin_memory()
    f = f_host.to(dev)
    grid = hzs.Grid(N, hzs.DIRICHLET, k=K_WAVE, nsub=NSUB, overlap=OVERLAP)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    def timed_solves(P, steps, warmup, e2e=False, **kw):
        u = torch.empty_like(f)
        u_host = torch.empty_like(f_host).pin_memory()
        for _ in range(warmup):
            P.solve(f, TOL, MAXIT, out=u, **kw)
        barrier()
        infos = []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            if e2e:
                fd = f_host.to(dev, non_blocking=True)
                _, inf = P.solve(fd, TOL, MAXIT, out=u, **kw)
                u_host.copy_(u, non_blocking=True)
            else:
                _, inf = P.solve(f, TOL, MAXIT, out=u, **kw)
            infos.append(inf[0])
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), world, dev), infos

    def arm(P, steps, warmup, note, **kw):
        ms, infos = timed_solves(P, steps, warmup, **kw)
        i0 = infos[-1]
        d = {"value": replica_throughput(len(infos), ms, world), "unit": "solves/s", "ms_per_step": ms / len(infos),
             "iterations": i0.iterations, "relres_est": i0.relres_est, "relres_true": i0.relres_true,
             "basis_bits": i0.basis_bits, "orth_kind": i0.orth_kind, "note": note}
        if kw.get("profile"):
            d.update({"t_precond_ms": i0.t_precond_ms, "t_matvec_ms": i0.t_matvec_ms, "t_orth_ms": i0.t_orth_ms,
                      "t_orth_dot_ms": i0.t_orth_dot_ms, "t_orth_update_ms": i0.t_orth_update_ms})
        return d, infos

    g_kw = {"graph": args.graph}
    # ---- mixed (headline)
    t0 = time.perf_counter()
    Pm = hzs.Preconditioner(grid, hzs.SHS2, hzs.COARSE_B2, P_COARSE, hzs.MIXED,
                            autotune=0 if args.no_autotune else 1)
    torch.cuda.synchronize()
    setup_mixed_s = time.perf_counter() - t0
    shape = Pm.info()
    clk = ClockSampler(local)
    clk.start()
    ms_tot, infos_plain = timed_solves(Pm, args.steps, args.warmup, **g_kw)
    clocks = clk.stop()
    # the same solves with CUDA events around every launch: phase times and the roofline
    nprof = max(2, args.steps // 4)
    ms_prof, infos = timed_solves(Pm, nprof, 0, profile=True)
    issue_alt = None
    if not args.no_alt_arm:
        issue_alt, _ = arm(Pm, max(2, args.steps // 4), 1, "stream launches" if args.graph else
                           "CUDA graphs of 8 Arnoldi steps", graph=not args.graph)
    ms_e2e, _ = timed_solves(Pm, max(2, args.steps // 2), 0, e2e=True, **g_kw)
    alt = {}
    if not args.no_alt_orth:
        alt["orth_dfma"], _ = arm(Pm, 2, 1, "the same delayed CGS2 with every FP64-accurate sum in FP64 FMAs on a "
                                  "complex128 basis (no FP32-pipe share)", orth_dfma=True, profile=True)
        alt["basis_df_32"], _ = arm(Pm, 2, 1, "delayed CGS2 on a double-float basis with bf16 remainders (about 32 "
                                    "bits), complex64 dot products: not an FP64 Arnoldi", basis_df=True, profile=True)
        alt["basis_df_48"], _ = arm(Pm, 2, 1, "delayed CGS2 on a double-float basis with complex64 remainders "
                                    "(about 48 bits), complex64 dot products: not an FP64 Arnoldi", basis_df=True,
                                    wide_basis=True, profile=True)
    Pm.close()
    dedup_off = None
    if not args.no_dedup_arm:
        Pn = hzs.Preconditioner(grid, hzs.SHS2, hzs.COARSE_B2, P_COARSE, hzs.MIXED, dedup_tiles=False)
        dedup_off, _ = arm(Pn, 2, 1, "every subdomain factor stored and streamed separately (no sharing of "
                           "identical factors)", profile=True)
        Pn.close()
    fp64 = None
    if not args.no_fp64:
        t0 = time.perf_counter()
        Pd = hzs.Preconditioner(grid, hzs.SHS2, hzs.COARSE_B2, P_COARSE, hzs.FP64)
        torch.cuda.synchronize()
        setup_fp64_s = time.perf_counter() - t0
        fp64, _ = arm(Pd, 2, 1, "complex128 throughout, classical CGS2 in FP64", profile=True)
        fp64["setup_s"] = setup_fp64_s
        Pd.close()
    grid.close()
    workloads = None
    if not args.no_workloads:
        workloads = other_configs(args, dev)
        b = batched_set(args, dev, args.graph)
        workloads["batched_mp2"] = {
            "value": replica_throughput(b["solves"], b["ms"], world), "unit": "solves/s", "ms_per_set": b["ms"],
            "e2e_value": replica_throughput(b["solves"], b["ms_e2e"], world), "setup_s": b["setup_s"],
            "problems": b["problems"],
            "note": "4 problems x 64 point sources at seeded nodes, solved concurrently (one stream per problem, "
                    "right-hand sides of a problem in lockstep)"}
    gpu_line_and_print(args, world, rank, locals())


def gpu_line_and_print(args, world, rank, L):
    """Assembles the JSON line of the GPU arm from the measurements in L."""
    import torch
    infos, infos_plain, pipes = L["infos"], L["infos_plain"], L["pipes"]
    last = infos[-1]
    it = last.iterations
    Nu = (N - 2) ** 2
    # ---- roofline of the two basis passes of the delayed CGS2 on the f53 basis (16 B a
    # basis entry: FP32 heads + 29-bit tails).  Algorithmic HBM bytes at step j:
    #   dot pass:    basis vectors 0..j-1, u~_j and w (16 (j + 2) Nu)
    #   update pass: basis vectors 0..j-1 (16 j Nu), u~_j and w read and written (64 Nu)
    # Step j = it completes the last column (dot pass only; its update returns at once).
    dot_bytes = sum(16 * (j + 2) * Nu for j in range(it + 1))
    upd_bytes = sum(16 * (j + 4) * Nu for j in range(it))
    t_dot = statistics.mean(i.t_orth_dot_ms for i in infos) * 1e-3
    t_upd = statistics.mean(i.t_orth_update_ms for i in infos) * 1e-3
    orth_s = statistics.mean(i.t_orth_ms for i in infos) * 1e-3
    peaks = _peaks_file()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = ("MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)" if "hbm_gbs" in peaks
                else "fallback 6800 GB/s")
    # FP64-accurate multiply-adds of a pass: 4 real multiply-adds (8 flops) per basis entry for
    # alpha (dot pass) or for sum c_i V_i (update pass), shared between the FP64 FMAs and the
    # FP32 error-free arithmetic; reported against the measured FP64 FMA rate
    macs = 8.0 * sum(j * Nu for j in range(it + 1))

    def pass_roofline(name, nbytes, t, nl, ratio):
        a = nbytes / t / 1e9 if t > 0 else 0.0
        tuned = any(k.startswith("HZS_F53_") for k in os.environ)
        return {"kernel": name, "bound": "hbm", "achieved": a, "peak": hbm_peak, "unit": "GB/s",
                "frac": a / hbm_peak, "traffic": None if tuned else ratio * nbytes / nl,
                "traffic_source": ("HZS_F53_* set: not the captured kernel version" if tuned else
                                   f"ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel at this size "
                                   f"(step j = 200: {ratio:.3f} x its algorithmic bytes), scaled to the average "
                                   f"launch's algorithmic bytes"),
                "peak_source": peak_src + ", of measured", "bytes_per_solve": nbytes, "time_per_solve_s": t,
                "launches": nl, "bytes_per_launch": nbytes / nl,
                "fp64_equivalent_tflops": macs / t / 1e12 if t > 0 else 0.0,
                "fp64_fma_peak_tflops": pipes["fp64_tflops"],
                "timing": "CUDA events around every launch of the kernel on the solve stream"}
    r_dot = pass_roofline("k_s53_dot_ws (delayed CGS2 dot pass on the f53 basis: FP64-accurate alpha, complex64 b)",
                          dot_bytes, t_dot, it + 1, TRAFFIC_RATIO["dot"])
    r_upd = pass_roofline("k_s53_update2 (delayed CGS2 update pass on the f53 basis, FP64-accurate, two entries "
                          "per thread)",
                          upd_bytes, t_upd, it, TRAFFIC_RATIO["update"])
    roofline = dict(r_upd if t_upd >= t_dot else r_dot)
    roofline["other_pass"] = r_dot if t_upd >= t_dot else r_upd
    roofline["orth_group"] = {"time_per_solve_s": orth_s, "achieved_gbs": (dot_bytes + upd_bytes) / orth_s / 1e9,
                              "note": "both passes plus the reduction, Givens, encode and scale kernels"}
    fp64 = L["fp64"]
    if fp64 is not None:
        # all-FP64 CGS2: 4 passes x (j+1) Nu complex multiply-adds (8 flops each) on the FP64 pipe
        it64 = fp64["iterations"]
        flops64 = sum(32.0 * (j + 1) * Nu for j in range(it64))
        t64 = fp64["t_orth_ms"] * 1e-3
        fp64["roofline"] = {"kernel": "CGS2 orthogonalisation, FP64 (k_multidot<double2> + k_axpy_multi)",
                            "bound": "alu", "achieved": flops64 / t64 / 1e12, "peak": pipes["fp64_tflops"],
                            "unit": "TFLOP/s", "frac": flops64 / t64 / 1e12 / pipes["fp64_tflops"],
                            "peak_source": "hzs_pipe_peaks FP64 FMA rate measured in this run, of measured"}
    world_ = world
    steps = args.steps
    value = replica_throughput(steps, L["ms_tot"], world_)
    i_last = infos_plain[-1]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world_, "steps": steps,
        "warmup": args.warmup, "ms_per_step": L["ms_tot"] / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("c64 preconditioner (stencil, transfers, subdomain solves); f64 coarse solve, outer operator, "
                  "Arnoldi basis (" + basis_dtype(i_last.basis_bits, i_last.orth_kind) + "), FP64-accurate "
                  "reorthogonalisation and update, f64 Hessenberg least squares and solution"),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "mixed", "n": N, "k": K_WAVE, "nsub": NSUB,
                   "overlap": OVERLAP, "coarse_ratio": P_COARSE, "tol": TOL, "basis_bits": i_last.basis_bits,
                   "l2": "working set larger than L2 (Krylov basis ~6 GB); no flush needed",
                   "issue": "CUDA graphs of 8 Arnoldi steps" if args.graph else "stream launches",
                   "parallelism": f"replicas x{world_}"},
        "iterations": i_last.iterations, "relres_est": i_last.relres_est, "relres_true": i_last.relres_true,
        "setup_s": L["setup_mixed_s"], "subdomain_solve_shape": L["shape"],
        "profiled": {"value": replica_throughput(len(infos), L["ms_prof"], world_), "unit": "solves/s",
                     "note": "solves with CUDA events around every launch (phases and roofline)"},
        "issue_alt": L["issue_alt"],
        "phases_ms": {"precond": last.t_precond_ms, "matvec": last.t_matvec_ms, "orth": last.t_orth_ms,
                      "orth_dot": last.t_orth_dot_ms, "orth_update": last.t_orth_update_ms,
                      "solve": last.t_solve_ms},
        "roofline": roofline,
        "e2e": {"value": replica_throughput(max(2, steps // 2), L["ms_e2e"], world_), "unit": "solves/s",
                "h2d_bytes_per_step": N * N * 16, "d2h_bytes_per_step": N * N * 16},
        "gpu_launches": int(sum(i.launches for i in infos_plain)),
        "clocks": L["clocks"],
        "pipe_peaks": pipes,
        "fp64": fp64,
        "orthogonalisations": L["alt"],
        "dedup_off": L["dedup_off"],
        "workloads": L["workloads"],
    }
    child = L["child"]
    if child is not None:
        res, why = finish_oracle_child(child, 600.0)
        if res is not None:
            line["cpu_baseline"] = {
                "value": 1.0 / res["t_solve_s"], "unit": "solves/s", "cores": 1, "kind": "oracle",
                "sample": (f"one complete solve of this workload by the FP64 oracle (numpy/scipy, SuperLU local "
                           f"solves, modified Gram-Schmidt GMRES) on one host core: {res['iterations']} steps in "
                           f"{res['t_solve_s']:.1f} s after a {res['t_setup_s']:.1f} s set-up; SuperLU solves hold "
                           "Python's GIL, so threads over the subdomains do not help"),
                "detail": res}
        else:
            line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": why}
    if world_ > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def batched_arm(args, world, rank, local):
    """The batched MP-2 set as its own line (one step = the whole set)."""
    import torch

    from paper_2408_03571_gb300 import build, hzs

    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    hzs.load()
    dev = torch.device("cuda", local)
    runs = [batched_set(args, dev, args.graph) for _ in range(max(1, args.steps))]
    ms = max_over_ranks(sum(r["ms"] for r in runs), world, dev)
    ms_e2e = max_over_ranks(sum(r["ms_e2e"] for r in runs), world, dev)
    nsol = sum(r["solves"] for r in runs)
    if rank != 0:
        return
    line = {
        "metric": "batched MP-2 Helmholtz solves/s to rel. residual 1e-6 (4 problems x %d right-hand sides)"
                  % args.nrhs,
        "value": replica_throughput(nsol, ms, world), "unit": "solves/s", "n_gpus": world, "steps": len(runs),
        "warmup": 1, "ms_per_step": ms / len(runs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 preconditioner; FP64 Arnoldi (f53 basis); f64 Hessenberg",
        "data": "synthetic",
        "config": {"workload": "MP-2 batch: (k, n) = (25, 257), (50, 257), (100, 513), (200, 1025), 64-node "
                               "subdomains, overlap 2, SHS2 with B2 and H = the largest 2^m h with kH <= 1, point "
                               "sources at seeded nodes, all problems concurrently",
                   "issue": "CUDA graphs of 8 Arnoldi steps" if args.graph else "stream launches",
                   "l2": "working set larger than L2; no flush needed", "parallelism": f"replicas x{world}"},
        "problems": runs[-1]["problems"], "setup_s": runs[-1]["setup_s"],
        "e2e": {"value": replica_throughput(nsol, ms_e2e, world), "unit": "solves/s",
                "h2d_bytes_per_step": runs[-1]["bytes_io"], "d2h_bytes_per_step": runs[-1]["bytes_io"]},
    }
    print(json.dumps(line), flush=True)


def profile_solve(args):
    """One MIXED solve of the workload, stream-issued (every kernel a plain launch), after set-up."""
    import numpy as np
    import torch

    from paper_2408_03571_gb300 import build, hzs
    from paper_2408_03571_gb300.inputs import point_source, random_source_nodes

    build.build()
    hzs.load()
    if args.workload == "batched":
        # one problem of the batched MP-2 set: H = p h, sources at seeded nodes as in the set
        g = hzs.Grid(N, hzs.SOMMERFELD, k=K_WAVE, nsub=NSUB, overlap=OVERLAP)
        P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, P_COARSE, hzs.MIXED)
        nodes = random_source_nodes(N, args.nrhs, 1000)
        F = torch.from_numpy(np.stack([point_source(N, nd) for nd in nodes])).cuda()
        P.solve(F, TOL, MAXIT)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        _, inf = P.solve(F, TOL, MAXIT)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"workload": f"MP-2 Sommerfeld, k={K_WAVE:g}, n={N}, {NSUB}x{NSUB} subdomains, overlap 2, "
                                      f"SHS2 with B2 H={P_COARSE}h, {args.nrhs} point sources, GMRES to 1e-6 "
                                      f"(at most {MAXIT} steps; profiling instance)",
                          "iterations_max": max(r.iterations for r in inf), "info": P.info()}), flush=True)
        P.close()
        g.close()
        return
    f = torch.from_numpy(point_source(N)).cuda()
    g = hzs.Grid(N, hzs.DIRICHLET, k=K_WAVE, nsub=NSUB, overlap=OVERLAP)
    P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, P_COARSE, hzs.MIXED)
    torch.cuda.synchronize()
    _, inf = P.solve(f, TOL, MAXIT)
    torch.cuda.synchronize()
    print(json.dumps({"workload": WORKLOAD, "iterations": inf[0].iterations, "launches": inf[0].launches,
                      "relres_true": inf[0].relres_true}), flush=True)
    P.close()
    g.close()


def main():
    args = parse()
    args.graph = not args.stream
    if args.oracle_full_solve:
        oracle_full_solve()
        return
    world, rank, local = dist_setup(args)
    if args.profile_solve:
        profile_solve(args)
        return
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    if args.workload == "batched":
        batched_arm(args, world, rank, local)
        return
    gpu_arm(args, world, rank, local)


if __name__ == "__main__":
    main()
