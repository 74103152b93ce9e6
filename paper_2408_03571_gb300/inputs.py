"""Seeded synthetic inputs shared, as data, by the CUDA path and the CPU oracle.

This module holds none of the solver's arithmetic: it only draws and lays out
the right-hand sides, wavenumber fields, receiver sets and random test vectors
that both sides consume.  Every array is on the host (numpy); callers move it
where they need it.

Layout convention (both sides): a grid function on the ``n x n`` uniform grid
of the unit square (mesh size ``h = 1/(n-1)``, Section 2) is a C-contiguous
``(n, n)`` array indexed ``[j, i]`` with ``i`` the x index and ``j`` the y
index, i.e. flat index ``j*n + i``.

Model problems (Section 2):
  * MP-1: Dirichlet boundary, unknowns are the ``(n-2)^2`` interior nodes.
  * MP-2: Sommerfeld boundary, unknowns are all ``n^2`` nodes.
The point source of Eq. (1) is discretised as ``1/h^2`` at one node; the model
problems put it at the centre ``(1/2, 1/2)``, which is a grid node for odd n.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "point_source",
    "centre_node",
    "random_source_nodes",
    "gaussian_bump_field",
    "kappa_field",
    "distinct_interior_nodes",
    "random_complex_grid",
]


def centre_node(n: int) -> tuple[int, int]:
    """(i, j) of the grid node at (1/2, 1/2); requires odd n."""
    if n % 2 != 1:
        raise ValueError("n must be odd so that (1/2, 1/2) is a grid node")
    c = (n - 1) // 2
    return c, c


def point_source(n: int, node: tuple[int, int] | None = None) -> np.ndarray:
    """Discrete Dirac delta of Eq. (1): ``1/h^2`` at ``node`` (default centre), complex128 (n, n)."""
    h = 1.0 / (n - 1)
    i, j = centre_node(n) if node is None else node
    f = np.zeros((n, n), dtype=np.complex128)
    f[j, i] = 1.0 / (h * h)
    return f


def random_source_nodes(n: int, count: int, seed: int, margin: int = 1) -> list[tuple[int, int]]:
    """``count`` seeded uniform-random nodes at least ``margin`` nodes inside the boundary."""
    rng = np.random.default_rng(seed)
    lo, hi = margin, n - margin  # hi exclusive
    ii = rng.integers(lo, hi, size=count)
    jj = rng.integers(lo, hi, size=count)
    return [(int(a), int(b)) for a, b in zip(ii, jj)]


def gaussian_bump_field(n: int, seed: int, nbumps: int = 16, width: float = 0.05) -> np.ndarray:
    """Seeded sum of Gaussian bumps on the grid, normalised to max |g| = 1.

    ``g(x, y) = sum_b a_b exp(-|(x, y) - c_b|^2 / (2 width^2))`` with centres
    ``c_b ~ U[0,1]^2`` and amplitudes ``a_b ~ U[-1, 1]``; returned as (n, n) float64.
    """
    rng = np.random.default_rng(seed)
    centres = rng.random((nbumps, 2))
    amps = rng.uniform(-1.0, 1.0, size=nbumps)
    x = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")  # X[j, i] = x_i, Y[j, i] = y_j
    g = np.zeros((n, n), dtype=np.float64)
    for (cx, cy), a in zip(centres, amps):
        g += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * width * width))
    m = np.max(np.abs(g))
    return g / m if m > 0 else g


def kappa_field(n: int, k0: float, seed: int, contrast: float = 0.2,
                perturb_seed: int | None = None, perturb: float = 0.25) -> np.ndarray:
    """Heterogeneous squared wavenumber ``kappa = (k0 (1 + contrast g))^2`` on the grid.

    With ``perturb_seed`` the bump field is ``normalise(g + perturb * g')`` with an
    independently seeded ``g'`` (used to make a target field near ``g``).
    """
    g = gaussian_bump_field(n, seed)
    if perturb_seed is not None:
        g = g + perturb * gaussian_bump_field(n, perturb_seed)
        g = g / np.max(np.abs(g))
    return (k0 * (1.0 + contrast * g)) ** 2


def distinct_interior_nodes(n: int, count: int, seed: int, margin: int = 1) -> list[tuple[int, int]]:
    """``count`` distinct seeded nodes at least ``margin`` inside the boundary."""
    rng = np.random.default_rng(seed)
    m = n - 2 * margin
    flat = rng.choice(m * m, size=count, replace=False)
    return [(int(margin + f % m), int(margin + f // m)) for f in flat]


def random_complex_grid(n: int, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Seeded complex128 grid function(s) with entries ``N(0,1) + i N(0,1)``."""
    rng = np.random.default_rng(seed)
    shape = (n, n) if nrhs is None else (nrhs, n, n)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
