"""The paper-table drivers (paper_2408_03571_gb300/tables.py) run the configurations
Section 5 prints (host logic only; no GPU):

* the first two tables: kappa_h = k h = 0.25 and H_sub = H = 4h give the grid, subdomain
  and coarse-grid counts of tests/golden/grid_counts.txt, and the overlap of 2 node
  layers is the largest that keeps every node in at most 4 subdomains;
* the k-n tables: the k and n axes of tests/golden/kn_sweep_axes.txt, and every n there
  admits H_sub = H = r h (r divides n - 1) with overlap r / 2.
"""
import os

from paper_2408_03571_gb300 import tables

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_regime_matches_tables_1_2():
    for line in _rows("grid_counts.txt"):
        nsub_total, Gh, GH, inv_h, inv_H, k = (int(t) for t in line.split())
        n, nsub, ov, p = tables.regime(k)
        assert n == inv_h + 1 and n * n == Gh
        assert nsub * nsub == nsub_total
        assert p == inv_h // inv_H and ((n - 1) // p + 1) ** 2 == GH
        w = (n - 1) // nsub                     # owned nodes per subdomain and axis: H_sub / h
        assert w == 4 and 2 * ov == w           # the largest overlap with <= 2 subdomains per axis


def test_kn_grid_matches_tables_3_4():
    for line in _rows("kn_sweep_axes.txt"):
        r, ks, ns = (part.split() for part in line.split("|"))
        r = int(r[0])
        ks_g, ns_g = tables.KN_GRID[r]
        assert [float(k) for k in ks] == [float(k) for k in ks_g]
        assert [int(n) for n in ns] == list(ns_g)
        for n in ns_g:
            assert (n - 1) % r == 0
