"""Oracle: overlapping subdomains, R_i and D_i (Section 3).

TEST INFRASTRUCTURE ONLY (FP64 CPU restatement, no code shared with the CUDA path).

Section 3 starts from a nonoverlapping decomposition of the square into N
pieces, extends each piece "by layers of grid nodes" to an overlapping
subdomain Omega_i, takes R_i as the 0/1 restriction to Omega_i, and asks for
diagonal D_i with sum_i R_i^T D_i R_i = I.  The paper does not fix the details;
this oracle reads them as follows (the CUDA path takes the same readings):

* square pieces: ``ns x ns`` blocks; per axis block ``a`` owns grid nodes
  ``[a w, (a+1) w)`` with ``w = (n-1)/ns``; the last block also owns node n-1;
* owned nodes are intersected with the unknowns (MP-1 drops the boundary);
* ``overlap`` = number of node layers added on each side of the owned block,
  clipped to the unknowns, so neighbouring subdomains share 2*overlap layers;
* D_i = 1 on the nodes subdomain i owns, 0 on its overlap (the restricted
  additive Schwarz choice); this satisfies sum_i R_i^T D_i R_i = I.
  Alternative reading (``scaling="multiplicity"``): D_i = 1/m(x) on every node x
  of subdomain i, m(x) the number of subdomains that contain x; it satisfies the
  same identity.
* the subdomain grid may be rectangular: ``ns`` is the count per axis or a pair
  (ns_x, ns_y).
"""
from __future__ import annotations

import numpy as np


def axis_blocks(n: int, ns: int, lo: int, hi: int, overlap: int):
    """Per-axis (owned_lo, owned_hi, ext_lo, ext_hi), inclusive unknown indices."""
    if (n - 1) % ns != 0:
        raise ValueError("ns must divide n-1")
    w = (n - 1) // ns
    if overlap < 0:
        raise ValueError("overlap must be >= 0")
    out = []
    for a in range(ns):
        o_lo = a * w
        o_hi = (a + 1) * w - 1 if a < ns - 1 else n - 1
        o_lo, o_hi = max(o_lo, lo), min(o_hi, hi)
        if o_lo > o_hi:
            raise ValueError("empty subdomain")
        e_lo, e_hi = max(o_lo - overlap, lo), min(o_hi + overlap, hi)
        out.append((o_lo, o_hi, e_lo, e_hi))
    return out


class Subdomain:
    def __init__(self, prob, xb, yb):
        self.own_x = (xb[0], xb[1]); self.own_y = (yb[0], yb[1])
        self.ext_x = (xb[2], xb[3]); self.ext_y = (yb[2], yb[3])
        xs = np.arange(xb[2], xb[3] + 1)
        ys = np.arange(yb[2], yb[3] + 1)
        self.mx, self.my = len(xs), len(ys)
        J, I = np.meshgrid(ys, xs, indexing="ij")          # lexicographic, x fastest
        self.idx = prob.index(I.ravel(), J.ravel())          # R_i as an index list
        owned = ((I >= xb[0]) & (I <= xb[1]) & (J >= yb[0]) & (J <= yb[1])).ravel()
        self.d = owned.astype(np.float64)                   # diagonal of D_i


OWNER, MULTIPLICITY = "owner", "multiplicity"


class Decomposition:
    def __init__(self, prob, ns, overlap: int, scaling: str = OWNER):
        nsx, nsy = (ns, ns) if np.isscalar(ns) else ns
        if scaling not in (OWNER, MULTIPLICITY):
            raise ValueError(scaling)
        self.ns, self.overlap, self.scaling = (nsx, nsy), overlap, scaling
        bx = axis_blocks(prob.n, nsx, prob.lo, prob.hi, overlap)
        by = axis_blocks(prob.n, nsy, prob.lo, prob.hi, overlap)
        self.subs = [Subdomain(prob, bx[a], by[b]) for b in range(nsy) for a in range(nsx)]
        self.N = prob.N
        if scaling == MULTIPLICITY:
            mult = np.zeros(prob.N)
            for s in self.subs:
                mult[s.idx] += 1.0
            for s in self.subs:
                s.d = 1.0 / mult[s.idx]

    def restrict(self, s: Subdomain, v: np.ndarray) -> np.ndarray:
        return v[s.idx]

    def prolong_add(self, s: Subdomain, y: np.ndarray, out: np.ndarray, weighted: bool):
        """out += R_i^T (D_i y) if weighted else R_i^T y."""
        out[s.idx] += (s.d * y) if weighted else y
