"""GMRES step counts of the experiments of Section 5 on the GPU.

Sweep 1 (the paper's first two tables): kappa_h = k h = 0.25, subdomains of
H_sub = 4h with the largest overlap that keeps every node in at most 4
subdomains (2 node layers), coarse spacing H = 4h, point source at the centre,
relative tolerance 1e-7, at most 100 steps; AS2, SAS2 and SHS2 with the P_1 and
B_2 coarse spaces:

    python -m paper_2408_03571_gb300.tables --bc sommerfeld --k 20 40 60 80 100 120 140 200

Sweep 2 (the last two tables): SHS2 with B_2 on MP-1 over a grid of k and n,
H_sub = H = r h for r = 4 or 16, overlap r/2, at most 50 steps:

    python -m paper_2408_03571_gb300.tables --kn 4
    python -m paper_2408_03571_gb300.tables --kn 16

Everything runs through the C ABI (hzs.py); a coarse space above 4096 unknowns
is solved by the block-tridiagonal LU (hzs_coarse_solver AUTO), or, with
--coarse-ml nsub,overlap,ratio, by the multilevel coarse solve:

    python -m paper_2408_03571_gb300.tables --bc sommerfeld --k 40 --coarse-ml 5,2,2
"""
from __future__ import annotations

import argparse
import time

import torch

from . import hzs
from .inputs import point_source

KINDS = (("AS2", hzs.AS2), ("SAS2", hzs.SAS2), ("SHS2", hzs.SHS2))
COARSES = (("P1", hzs.COARSE_P1), ("B2", hzs.COARSE_B2))


def regime(k: float) -> tuple[int, int, int, int]:
    """(n, subdomains per axis, overlap, H/h) for kappa_h = 0.25 and H_sub = H = 4h."""
    n = 4 * int(round(k)) + 1
    return n, int(round(k)), 2, 4


def run(bc: int, ks, precision: int = hzs.FP64, tol: float = 1e-7, maxit: int = 100, device: int = 0,
        ml: tuple[int, int, int] | None = None):
    """List of rows {k, n, Nc, (name, coarse): (steps, converged, ms per solve)}.  ml: the
    multilevel coarse solve (coarse subdomains per axis, overlap, coarse-of-coarse ratio)
    in place of the exact one."""
    torch.cuda.set_device(device)
    rows = []
    for k in ks:
        n, nsub, ov, p = regime(k)
        g = hzs.Grid(n, bc, k=float(k), nsub=nsub, overlap=ov)
        f = torch.from_numpy(point_source(n)).cuda()
        row = {"k": k, "n": n}
        for cname, coarse in COARSES:
            for kname, kind in KINDS:
                kw = dict(coarse_solver=hzs.COARSE_SOLVER_MULTILEVEL, ml=ml) if ml else {}
                P = hzs.Preconditioner(g, kind, coarse, p, precision, **kw)
                P.solve(f, tol, maxit)                       # warm-up (work space, first launches)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, info = P.solve(f, tol, maxit)
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t0) * 1e3
                row[(kname, cname)] = (info[0].iterations, bool(info[0].converged), ms)
                P.close()
        g.close()
        rows.append(row)
    return rows


# (k values, n values) of the k-n sweeps for H_sub = H = 4h and 16h
KN_GRID = {
    4: ([10, 20, 30, 40, 50], list(range(33, 162, 8))),
    16: ([5, 10, 15, 20, 25, 30], list(range(33, 258, 16))),
}


def run_kn(ratio: int, ks, ns, precision: int = hzs.FP64, tol: float = 1e-7, maxit: int = 50, device: int = 0):
    """SHS2 / B_2 step counts on MP-1 with H_sub = H = ratio h, overlap ratio/2:
    {(k, n): (steps, converged)}."""
    torch.cuda.set_device(device)
    out = {}
    for n in ns:
        nsub = (n - 1) // ratio
        f = torch.from_numpy(point_source(n)).cuda()
        for k in ks:
            g = hzs.Grid(n, hzs.DIRICHLET, k=float(k), nsub=nsub, overlap=ratio // 2)
            P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, ratio, precision)
            _, info = P.solve(f, tol, maxit)
            out[(k, n)] = (info[0].iterations, bool(info[0].converged))
            P.close()
            g.close()
    return out


def format_kn(res, ks, ns) -> str:
    head = "| k \\ n | " + " | ".join(str(n) for n in ns) + " |"
    sep = "|" + "---|" * (1 + len(ns))
    lines = [head, sep]
    for k in ks:
        cells = [str(res[(k, n)][0]) if res[(k, n)][1] else "x" for n in ns]
        lines.append(f"| {k} | " + " | ".join(cells) + " |")
    return "\n".join(lines)


def format_rows(rows) -> str:
    head = "| k | n | " + " | ".join(f"{kn} {cn}" for cn, _ in COARSES for kn, _ in KINDS) + " |"
    sep = "|" + "---|" * (2 + len(COARSES) * len(KINDS))
    out = [head, sep]
    for r in rows:
        cells = []
        for cn, _ in COARSES:
            for kn, _ in KINDS:
                it, conv, _ = r[(kn, cn)]
                cells.append(str(it) if conv else "x")
        out.append(f"| {r['k']:g} | {r['n']} | " + " | ".join(cells) + " |")
    return "\n".join(out)


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--bc", choices=["dirichlet", "sommerfeld"], default="sommerfeld")
    ap.add_argument("--k", type=float, nargs="+", default=[20, 40, 60, 80, 100, 120, 140, 200])
    ap.add_argument("--mixed", action="store_true", help="complex64 preconditioner inside FP64 FGMRES")
    ap.add_argument("--kn", type=int, choices=[4, 16], help="the k-n sweep with H_sub = H = 4h or 16h")
    ap.add_argument("--coarse-ml", type=str, default=None,
                    help="multilevel coarse solve 'nsub,overlap,ratio' on the coarse grid instead of the exact one")
    args = ap.parse_args()
    hzs.load()
    prec = hzs.MIXED if args.mixed else hzs.FP64
    if args.kn:
        ks, ns = KN_GRID[args.kn]
        print(format_kn(run_kn(args.kn, ks, ns, prec), ks, ns))
        return
    bc = hzs.SOMMERFELD if args.bc == "sommerfeld" else hzs.DIRICHLET
    ml = tuple(int(x) for x in args.coarse_ml.split(",")) if args.coarse_ml else None
    rows = run(bc, args.k, prec, ml=ml)
    print(format_rows(rows))
    for r in rows:
        t = sum(v[2] for key, v in r.items() if isinstance(key, tuple))
        print(f"k={r['k']:g}: {t:.1f} ms for the 6 solves")


if __name__ == "__main__":
    main()
