"""The seeded synthetic inputs have the shapes and distributions the workloads state:

* the point source is 1/h^2 at one node (the centre by default): Eq. 1's delta source
  at (1/2, 1/2) discretised as the grid function of unit integral;
* source nodes, receivers and finite-difference nodes are seeded, inside the boundary
  by the requested margin, and distinct where asked;
* the bump field is a sum of 16 Gaussians normalised to max |g| = 1, so
  kappa = (k0 (1 + 0.2 g))^2 stays within [(0.8 k0)^2, (1.2 k0)^2] and reaches an end;
* the target field's perturbation keeps the same bounds and differs from the field;
* every generator returns the same arrays for the same seed.
"""
import numpy as np

from paper_2408_03571_gb300 import inputs


def test_point_source():
    n = 33
    f = inputs.point_source(n)
    h = 1.0 / (n - 1)
    assert f.dtype == np.complex128 and f.shape == (n, n)
    assert np.count_nonzero(f) == 1 and f[16, 16] == 1.0 / h**2
    g = inputs.point_source(n, (3, 7))
    assert g[7, 3] == 1.0 / h**2 and np.count_nonzero(g) == 1


def test_seeded_nodes():
    n = 65
    a = inputs.random_source_nodes(n, 200, seed=5, margin=2)
    assert a == inputs.random_source_nodes(n, 200, seed=5, margin=2)
    assert all(2 <= i <= n - 3 and 2 <= j <= n - 3 for i, j in a)
    d = inputs.distinct_interior_nodes(n, 64, seed=9)
    assert len(set(d)) == 64 and all(1 <= i <= n - 2 and 1 <= j <= n - 2 for i, j in d)
    assert d != inputs.distinct_interior_nodes(n, 64, seed=10)


def test_kappa_field_bounds():
    n, k0 = 129, 100.0
    g = inputs.gaussian_bump_field(n, seed=2001)
    assert np.max(np.abs(g)) == 1.0
    kap = inputs.kappa_field(n, k0, seed=2001)
    assert kap.shape == (n, n) and np.all(kap > 0)
    k = np.sqrt(kap)
    assert k.min() >= 0.8 * k0 - 1e-9 and k.max() <= 1.2 * k0 + 1e-9
    assert np.isclose(k.min(), 0.8 * k0) or np.isclose(k.max(), 1.2 * k0)
    kt = np.sqrt(inputs.kappa_field(n, k0, seed=2001, perturb_seed=2002))
    assert kt.min() >= 0.8 * k0 - 1e-9 and kt.max() <= 1.2 * k0 + 1e-9
    assert not np.allclose(kt, k)
    assert np.array_equal(kap, inputs.kappa_field(n, k0, seed=2001))


def test_random_complex_grid():
    a = inputs.random_complex_grid(17, seed=3, nrhs=4)
    assert a.shape == (4, 17, 17) and a.dtype == np.complex128
    assert np.array_equal(a, inputs.random_complex_grid(17, seed=3, nrhs=4))
    b = inputs.random_complex_grid(257, seed=4)
    assert abs(b.real.std() - 1) < 0.02 and abs(b.imag.std() - 1) < 0.02 and abs(b.mean()) < 0.02
