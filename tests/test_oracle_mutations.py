"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle, on the CPU, and runs the pins that
should see it; at least one of them must fail. Most mistakes are planted by
editing one expression in the oracle's own source (the function is recompiled
from the edited text in its module's namespace). A few are planted at the level
of the matrix or function they spoil. Every plant is undone after its case.

A pin that lets a mistake through does not pin what it claims. So each kind of
slip is planted once: a flipped sign, a dropped term, a wrong scaling, a wrong
shift or width, a missing or misplaced complex conjugate, a wrong combination
of terms.

* Section 2 (Eqs. 1-3): Sommerfeld term with the wrong sign; edge rows not
  halved; the -kappa term dropped; neighbour couplings with the wrong sign;
  d A_PP / d kappa with the wrong sign or without its boundary part; the kappa
  field read with x and y swapped;
* Section 3: D_i = 1 on the whole subdomain; overlap added on one side only;
  local solves with conj(A_i);
* Section 4: B_2 shifted by half a cell; a wrong middle piece of the quadratic
  B-spline; P_1 hats twice as wide; MP-1 keeping its coarse boundary nodes;
  A_0 built from conj(A);
* Eqs. 4-6: SHS2 deflating with v + A Q v; SAS2 without D_i; AS2 without Q;
* Section 5: the Givens sine conjugated; the Gram-Schmidt inner product
  conjugated on the wrong side; the solution formed without M^{-1};
* the adjoint: the gradient's sign; the adjoint solved without the conjugate.
"""
import inspect
import textwrap

import numpy as np
import pytest
import scipy.sparse as sp

import importlib

import oracle as opkg
from oracle import AS1, AS2, B2, DIRICHLET, P1, SAS2, SHS2, SOMMERFELD, Problem

# the oracle's modules (the package re-exports a function named gmres, so each
# submodule is looked up by its full name)
oadj, ocoarse, odec, ogmres, oproblem, oschwarz = (
    importlib.import_module(f"oracle.{m}") for m in ("adjoint", "coarse", "decomposition", "gmres", "problem",
                                                      "schwarz"))

import test_oracle_coarse as tc
import test_oracle_problem as tp
import test_oracle_schwarz as ts


def mutant(func, *edits):
    """func recompiled from its source with each (old, new) text edit applied once."""
    src = textwrap.dedent(inspect.getsource(func))
    for old, new in edits:
        assert src.count(old) >= 1, (func.__name__, old)
        src = src.replace(old, new)
    ns = dict(func.__globals__)
    exec(compile(src, f"<mutant of {func.__qualname__}>", "exec"), ns)
    return ns[func.__name__]


def plant(mp, owner, name, *edits):
    """Replaces owner.name by its mutant, and every module-level reference to the same
    function that the oracle package and the pin modules imported by name."""
    orig = getattr(owner, name)
    new = mutant(orig, *edits)
    mp.setattr(owner, name, new)
    if inspect.ismodule(owner):
        for mod in (opkg, oproblem, ocoarse, odec, oschwarz, ogmres, oadj, tc, tp, ts):
            if getattr(mod, name, None) is orig:
                mp.setattr(mod, name, new)


def caught(pins) -> bool:
    """True if at least one (callable, args) pin fails one of its assertions (any other
    exception propagates: a mutant that cannot run has not been caught by a pin)."""
    for fn, args in pins:
        try:
            fn(*args)
        except AssertionError:
            return True
    return False


# ---- Section 2 ---------------------------------------------------------------------

def sommerfeld_sign(mp):
    plant(mp, Problem, "diag_entry", ("-k / h)", "k / h)"))
    plant(mp, Problem, "assemble_fast", ("diag = diag - 1j *", "diag = diag + 1j *"))
    return [(tp.test_sommerfeld_rows_consistent, ("right",)), (tp.test_sommerfeld_rows_consistent, ("corner",))]


def edge_rows_not_halved(mp):
    # the symmetrising row scaling forgotten: boundary rows keep their ghost-node weights
    for name in ("assemble", "assemble_fast"):
        orig = getattr(Problem, name)

        def doubled(self, _orig=orig):
            A = _orig(self).tocsr()
            s = np.ones(self.N)
            for j in range(self.lo, self.hi + 1):
                for i in range(self.lo, self.hi + 1):
                    if self.bc == SOMMERFELD and self.boundary_count(i, j) > 0:
                        s[self.index(i, j)] = 2.0 ** self.boundary_count(i, j)
            return sp.csr_matrix(sp.diags(s) @ A)
        mp.setattr(Problem, name, doubled)
    return [(tp.test_symmetry_and_realness, (9,))]


def kappa_dropped(mp):
    plant(mp, Problem, "diag_entry", ("4.0 / h**2 - kap", "4.0 / h**2"))
    plant(mp, Problem, "assemble_fast", ("np.where(nb == 0, 4.0 / h**2 - kap,", "np.where(nb == 0, 4.0 / h**2,"))
    return [(tp.test_interior_row_sums, ()), (tp.test_mp1_matches_sine_series, (17, 13.0))]


def coupling_sign(mp):
    plant(mp, Problem, "offdiag_entry", ("if self.bc == DIRICHLET:\n        return -1.0 / h**2",
                                         "if self.bc == DIRICHLET:\n        return 1.0 / h**2"))
    plant(mp, Problem, "assemble_fast", ("w = np.full(ii.shape, -1.0 / h**2)", "w = np.full(ii.shape, 1.0 / h**2)"))
    return [(tp.test_mp1_matches_sine_series, (17, 13.0))]


def dkappa_sign(mp):
    plant(mp, Problem, "ddiag_dkappa", ("return complex(-0.5, -dk / h)", "return complex(0.5, dk / h)"),
          ("return complex(-0.25, -dk / h)", "return complex(0.25, dk / h)"))
    return [(tp.test_dA_dkappa_matches_difference, ())]


def dkappa_no_boundary_part(mp):
    plant(mp, Problem, "ddiag_dkappa", ("return complex(-0.5, -dk / h)", "return complex(-1.0)"),
          ("return complex(-0.25, -dk / h)", "return complex(-1.0)"))
    return [(tp.test_dA_dkappa_matches_difference, ())]


def kappa_field_transposed(mp):
    plant(mp, Problem, "diag_entry", ("self.kappa[j, i]", "self.kappa[i, j]"))
    plant(mp, Problem, "ddiag_dkappa", ("self.kappa[j, i]", "self.kappa[i, j]"))
    plant(mp, Problem, "assemble_fast", ("kap = self.kappa[jj, ii]", "kap = self.kappa[ii, jj]"))
    return [(tp.test_dA_dkappa_matches_difference, ()), (tp.test_assembly_paths_agree, (SOMMERFELD, 9, True))]


# ---- Section 3 ---------------------------------------------------------------------

def d_is_identity(mp):
    plant(mp, odec.Subdomain, "__init__", ("self.d = owned.astype(np.float64)", "self.d = np.ones(owned.shape)"))
    return [(ts.test_partition_identity, (DIRICHLET, 2, 2))]


def overlap_one_sided(mp):
    plant(mp, odec, "axis_blocks", ("e_lo, e_hi = max(o_lo - overlap, lo)", "e_lo, e_hi = max(o_lo, lo)"))
    return [(ts.test_partition_identity, (SOMMERFELD, 4, 2)),
            (ts.test_overlap_is_layers_of_nodes_on_every_side, (SOMMERFELD, 4, 2))]


def local_solve_conjugated(mp):
    plant(mp, oschwarz.Schwarz, "local_sum",
          ("y = lu.solve(np.ascontiguousarray(r[s.idx], dtype=np.complex128))",
           "y = np.conj(lu.solve(np.conj(np.ascontiguousarray(r[s.idx], dtype=np.complex128))))"))
    return [(ts.test_preconditioner_dense_formula, (SOMMERFELD, AS1, B2))]


# ---- Section 4 ---------------------------------------------------------------------

def b2_half_cell_shift(mp):
    plant(mp, ocoarse, "basis_1d", ("bspline2((x - XI) / H + 1.5)", "bspline2((x - XI) / H + 1.0)"))
    return [(tc.test_b2_weights_h2_match_eq7, ())]


def b2_middle_piece(mp):
    plant(mp, ocoarse, "bspline2", ("6.0 * t[b] - 3.0", "6.0 * t[b] - 2.0"))
    return [(tc.test_b2_weights_h2_match_eq7, ()), (tc.test_partition_of_unity, (B2, 4))]


def p1_hat_too_wide(mp):
    plant(mp, ocoarse, "hat", ("1.0 - np.abs(t)", "1.0 - np.abs(t) / 2.0"))
    return [(tc.test_p1_interpolatory, ())]


def mp1_keeps_coarse_boundary(mp):
    plant(mp, ocoarse.CoarseSpace, "__init__", ("keep = prob.bc != DIRICHLET", "keep = True"))
    return [(tc.test_R0_is_tensor_product, (DIRICHLET, B2))]


def galerkin_of_conj(mp):
    plant(mp, ocoarse.CoarseSpace, "galerkin", ("self.R0 @ A @ self.R0.T", "self.R0 @ A.conj() @ self.R0.T"))
    return [(ts.test_preconditioner_dense_formula, (SOMMERFELD, SHS2, B2))]


# ---- Eqs. 4-6 ----------------------------------------------------------------------

def shs2_deflation_sign(mp):
    plant(mp, oschwarz.Schwarz, "apply", ("w = v - self.Ap @ q", "w = v + self.Ap @ q"))
    return [(ts.test_preconditioner_dense_formula, (DIRICHLET, SHS2, B2))]


def sas2_without_d(mp):
    plant(mp, oschwarz.Schwarz, "apply", ("z = q + self.local_sum(v, weighted=True)",
                                         "z = q + self.local_sum(v, weighted=False)"))
    return [(ts.test_preconditioner_dense_formula, (DIRICHLET, SAS2, P1))]


def as2_without_q(mp):
    plant(mp, oschwarz.Schwarz, "apply", ("z = q + self.local_sum(v, weighted=False)",
                                         "z = self.local_sum(v, weighted=False)"))
    return [(ts.test_preconditioner_dense_formula, (SOMMERFELD, AS2, B2))]


def c64_mode_in_fp64(mp):
    # the complex64 preconditioner silently computed in FP64
    plant(mp, oschwarz.Schwarz, "__init__", ("self.ct = np.complex128 if precision == FP64 else np.complex64",
                                            "self.ct = np.complex128"))
    return [(ts.test_complex64_preconditioner_is_the_same_operator_rounded, (DIRICHLET, SAS2))]


def c64_factors_transposed(mp):
    # the complex64 local solve with its triangular factors applied in the wrong order
    plant(mp, oschwarz.Schwarz, "_solve32", ("y = spla.spsolve_triangular(L, pb, lower=True, unit_diagonal=True)",
                                            "y = spla.spsolve_triangular(U, pb, lower=False)"),
          ("z = spla.spsolve_triangular(U, y, lower=False)",
           "z = spla.spsolve_triangular(L, y, lower=True, unit_diagonal=True)"))
    return [(ts.test_complex64_preconditioner_is_the_same_operator_rounded, (SOMMERFELD, AS1))]


def c64_coarse_solve_dropped(mp):
    plant(mp, oschwarz.Schwarz, "apply_Q", ("c = self.coarse.solve(c).astype(np.complex64)",
                                           "c = c.astype(np.complex64)"))
    return [(ts.test_complex64_preconditioner_is_the_same_operator_rounded, (SOMMERFELD, SHS2))]


def c64_deflation_with_other_transfer(mp):
    # the complex64 coarse correction prolongated with 1.001 R_0^T instead of R_0^T (a
    # prolongation that is not the restriction's transpose), so R_0 (v - A Q v) != 0
    plant(mp, oschwarz.Schwarz, "apply_Q", ("return self.R0p.T @ c",
                                           "return self.R0p.T @ c + 1e-3 * (self.R0p.T @ c)"))
    return [(ts.test_complex64_deflation_annihilates_the_coarse_residual, ())]


# ---- Section 5 ---------------------------------------------------------------------

def givens_sine_conjugated(mp):
    plant(mp, ogmres, "givens", ("return aa / rho, (a / aa) * np.conj(b) / rho", "return aa / rho, np.conj(a / aa) * b / rho"))
    return [(ts.test_gmres_minimal_residual_bruteforce, (SOMMERFELD,)), (ts.test_givens_rotation, ())]


def gram_schmidt_conjugate_side(mp):
    plant(mp, ogmres, "gmres", ("H[i, j] = np.vdot(V[i], w)", "H[i, j] = np.vdot(w, V[i])"))
    return [(ts.test_gmres_minimal_residual_bruteforce, (SOMMERFELD,))]


def solution_without_preconditioner(mp):
    plant(mp, ogmres, "gmres", ("x = M_apply(sum(y[i] * V[i] for i in range(m)))",
                                "x = sum(y[i] * V[i] for i in range(m))"))
    return [(ts.test_gmres_minimal_residual_bruteforce, (DIRICHLET,))]


# ---- adjoint -------------------------------------------------------------------------

def gradient_sign(mp):
    plant(mp, oadj, "kappa_gradient", ("return -np.real(", "return np.real("))
    return [(ts.test_adjoint_gradient_vs_finite_differences, (SOMMERFELD,))]


def adjoint_without_conjugate(mp):
    plant(mp, oadj, "adjoint_solve", ("M_apply, np.conj(g), tol, maxit)", "M_apply, g, tol, maxit)"),
          ("lam = np.conj(res.x)", "lam = res.x"))
    return [(ts.test_adjoint_gradient_vs_finite_differences, (SOMMERFELD,))]


MUTATIONS = [
    sommerfeld_sign, edge_rows_not_halved, kappa_dropped, coupling_sign, dkappa_sign,
    dkappa_no_boundary_part, kappa_field_transposed, d_is_identity, overlap_one_sided, local_solve_conjugated,
    b2_half_cell_shift, b2_middle_piece, p1_hat_too_wide, mp1_keeps_coarse_boundary, galerkin_of_conj,
    shs2_deflation_sign, sas2_without_d, as2_without_q, c64_mode_in_fp64, c64_factors_transposed, c64_coarse_solve_dropped,
    c64_deflation_with_other_transfer, givens_sine_conjugated,
    gram_schmidt_conjugate_side, solution_without_preconditioner, gradient_sign, adjoint_without_conjugate,
]


@pytest.mark.parametrize("plant_fn", MUTATIONS, ids=[m.__name__ for m in MUTATIONS])
def test_planted_mistake_is_caught(plant_fn, monkeypatch):
    pins = plant_fn(monkeypatch)
    assert caught(pins), f"no pin caught: {plant_fn.__name__}"


def test_pins_pass_on_the_oracle_as_written():
    """The same pin calls pass without a planted mistake, so each catch above is the mistake's."""
    pins = []
    for plant_fn in MUTATIONS:
        with pytest.MonkeyPatch.context() as mp:
            pins += plant_fn(mp)
    assert oproblem.Problem is Problem
    for fn, args in dict.fromkeys(pins):
        fn(*args)
