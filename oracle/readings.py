"""Oracle experiment: the k = 20 rows of the paper's first two tables (Section 5:
MP-2 and MP-1, kappa h = 0.25, H_sub = H = 4h, overlap 2, centre source, tol 1e-7,
at most 100 steps) under each reading the paper leaves open.

TEST INFRASTRUCTURE ONLY (runs the FP64 CPU oracle; prints a table).

Readings varied (the others as in the oracle's default):
  right / left   side of the preconditioner in GMRES (Section 5 does not say;
                 MATLAB's gmres applies a given preconditioner on the left)
  owner / mult   D_i of SAS2 and SHS2: owner indicator or 1/multiplicity (Section 3)
  spline / comp  B_2 for H = 4h: the quadratic B-spline of knot spacing H, or
                 Eq. (7)'s H = 2h operator composed twice
  ov2 / ov1      "overlap 2": node layers added on each side of an owned block
                 (neighbours share 4 layers), or layers shared by neighbours (one
                 added on each side)

Usage: python -m oracle.readings [k]
"""
from __future__ import annotations

import sys

from .coarse import B2, P1
from .gmres import gmres
from .problem import DIRICHLET, SOMMERFELD, Problem
from .schwarz import AS2, SAS2, SHS2, Schwarz

# printed counts at k = 20 (Table 1: MP-2, Table 2: MP-1), columns as COMBOS
PAPER_K20 = {SOMMERFELD: (21, 15, 9, 21, 16, 8), DIRICHLET: (21, 16, 9, 20, 14, 7)}
COMBOS = ((AS2, P1), (SAS2, P1), (SHS2, P1), (AS2, B2), (SAS2, B2), (SHS2, B2))
READINGS = (
    ("right/owner/spline/ov2", dict(side="right", scaling="owner", b2_mode="spline", ov=2)),
    ("left/owner/spline/ov2", dict(side="left", scaling="owner", b2_mode="spline", ov=2)),
    ("right/mult/spline/ov2", dict(side="right", scaling="multiplicity", b2_mode="spline", ov=2)),
    ("right/owner/comp/ov2", dict(side="right", scaling="owner", b2_mode="composed", ov=2)),
    ("right/owner/spline/ov1", dict(side="right", scaling="owner", b2_mode="spline", ov=1)),
    ("left/mult/spline/ov2", dict(side="left", scaling="multiplicity", b2_mode="spline", ov=2)),
    ("left/mult/spline/ov1", dict(side="left", scaling="multiplicity", b2_mode="spline", ov=1)),
    ("left/mult/comp/ov1", dict(side="left", scaling="multiplicity", b2_mode="composed", ov=1)),
)


def table_row(bc: str, k: float, reading: dict, maxit: int = 100, tol: float = 1e-7):
    """Step counts of the six combinations (None: the cap was reached)."""
    from paper_2408_03571_gb300.inputs import point_source

    n = int(round(k / 0.25)) + 1              # kappa h = 0.25
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast()
    f = prob.grid_to_vec(point_source(n))
    out = []
    for kind, coarse in COMBOS:
        M = Schwarz(prob, A, (n - 1) // 4, reading["ov"], kind, coarse, 4, scaling=reading["scaling"],
                    b2_mode=reading["b2_mode"])
        r = gmres(lambda x: A @ x, M.apply, f, tol, maxit, side=reading["side"])
        out.append(r.iterations if r.converged else None)
    return out


def main(argv):
    k = float(argv[1]) if len(argv) > 1 else 20.0
    fmt = lambda v: "x" if v is None else str(v)
    for bc, name in ((SOMMERFELD, "MP-2"), (DIRICHLET, "MP-1")):
        print(f"{name}, k = {k:g}: AS2 P1 | SAS2 P1 | SHS2 P1 | AS2 B2 | SAS2 B2 | SHS2 B2")
        if k == 20.0:
            print(f"  {'paper':24s}", " | ".join(fmt(v) for v in PAPER_K20[bc]))
        for label, rd in READINGS:
            print(f"  {label:24s}", " | ".join(fmt(v) for v in table_row(bc, k, rd)), flush=True)


if __name__ == "__main__":
    main(sys.argv)
