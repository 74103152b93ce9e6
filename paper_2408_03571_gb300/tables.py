"""GMRES step counts in the H_sub = H = 4h regime of Section 5 (the paper's first
two tables): kappa_h = k h = 0.25, subdomains of 4h with the largest overlap
that keeps every node in at most 4 subdomains (2 node layers), coarse spacing
H = 4h, point source at the centre, relative tolerance 1e-7, at most 100 steps.

    python -m paper_2408_03571_gb300.tables --bc sommerfeld --k 20 40 60 80 100 120 140 200

prints, per k, the step counts of AS2, SAS2 and SHS2 with the P_1 and B_2
coarse spaces and the GPU time per solve.  Everything runs through the C ABI
(hzs.py); a coarse space above 4096 unknowns is solved by the block-tridiagonal
LU (hzs_coarse_solver AUTO).
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


def run(bc: int, ks, precision: int = hzs.FP64, tol: float = 1e-7, maxit: int = 100, device: int = 0):
    """List of rows {k, n, Nc, (name, coarse): (steps, converged, ms per solve)}."""
    torch.cuda.set_device(device)
    rows = []
    for k in ks:
        n, nsub, ov, p = regime(k)
        g = hzs.Grid(n, bc, k=float(k), nsub=nsub, overlap=ov)
        f = torch.from_numpy(point_source(n)).cuda()
        row = {"k": k, "n": n}
        for cname, coarse in COARSES:
            for kname, kind in KINDS:
                P = hzs.Preconditioner(g, kind, coarse, p, precision)
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
    args = ap.parse_args()
    hzs.load()
    bc = hzs.SOMMERFELD if args.bc == "sommerfeld" else hzs.DIRICHLET
    rows = run(bc, args.k, hzs.MIXED if args.mixed else hzs.FP64)
    print(format_rows(rows))
    for r in rows:
        t = sum(v[2] for key, v in r.items() if isinstance(key, tuple))
        print(f"k={r['k']:g}: {t:.1f} ms for the 6 solves")


if __name__ == "__main__":
    main()
