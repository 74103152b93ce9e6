"""Oracle experiment: outer step counts with the multilevel coarse solve (SHS2 on the
coarse grid G_H in place of A_0^{-1}; Section 5 names the exact coarse solve as the
cost that grows with |G_H|), in the setting of the paper's first two tables (kappa h =
0.25, H_sub = H = 4h, overlap 2, centre point source, tol 1e-7, at most 100 steps).

TEST INFRASTRUCTURE ONLY (runs the FP64 CPU oracle; prints a table).

Columns: the exact coarse solve; one application of SHS2 on G_H (ns0 coarse subdomains
per axis, overlap 2, coarse-of-coarse ratio p0); inner right-preconditioned GMRES on
A_0 with that SHS2 to a relative tolerance (outer flexible GMRES), with the mean inner
steps per coarse solve in brackets.

Usage: python -m oracle.multilevel_study [k ...]
"""
from __future__ import annotations

import sys

import numpy as np

from .coarse import B2
from .gmres import gmres
from .problem import DIRICHLET, SOMMERFELD, Problem
from .schwarz import SHS2, Schwarz

VARIANTS = (("once ns0=5 p0=2", dict(ns=5, ov=2, p=2)), ("once ns0=5 p0=4", dict(ns=5, ov=2, p=4)),
            ("once ns0=2 p0=2", dict(ns=2, ov=2, p=2)), ("inner 1e-1", dict(ns=5, ov=2, p=2, inner_tol=1e-1)),
            ("inner 1e-2", dict(ns=5, ov=2, p=2, inner_tol=1e-2)), ("inner 1e-4", dict(ns=5, ov=2, p=2, inner_tol=1e-4)),
            ("inner 1e-8", dict(ns=5, ov=2, p=2, inner_tol=1e-8)))


def row(bc: str, k: float, tol: float = 1e-7, maxit: int = 100):
    """[(label, outer steps or None, mean inner steps)] for one (bc, k)."""
    from paper_2408_03571_gb300.inputs import point_source

    n = int(round(k / 0.25)) + 1
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast()
    f = prob.grid_to_vec(point_source(n))
    ns = (n - 1) // 4
    ref = gmres(lambda x: A @ x, Schwarz(prob, A, ns, 2, SHS2, B2, 4).apply, f, tol, maxit)
    out = [("exact", ref.iterations if ref.converged else None, 0.0)]
    for label, cs in VARIANTS:
        M = Schwarz(prob, A, ns, 2, SHS2, B2, 4, coarse_solve=cs)
        r = gmres(lambda x: A @ x, M.apply, f, tol, maxit, flexible="inner_tol" in cs)
        its = M.coarse.inner.inner_its
        out.append((label, r.iterations if r.converged else None, float(np.mean(its)) if its else 0.0))
    return out


def main(argv):
    ks = [float(a) for a in argv[1:]] or [40.0]
    for bc, name in ((SOMMERFELD, "MP-2"), (DIRICHLET, "MP-1")):
        for k in ks:
            cells = [f"{lab}: {'x' if it is None else it}" + (f" ({inner:.1f})" if inner else "")
                     for lab, it, inner in row(bc, k)]
            print(f"{name} k={k:g}: " + " | ".join(cells), flush=True)


if __name__ == "__main__":
    main(sys.argv)
