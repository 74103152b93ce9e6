"""FP64 CPU oracle for two-level Schwarz preconditioned GMRES on 2-D Helmholtz.

TEST INFRASTRUCTURE ONLY.  This package restates the method of "Coarse Spaces
Based on Higher-Order Interpolation for Schwarz Preconditioners for Helmholtz
Problems" (Sections 2-5) plainly and slowly in FP64 on the CPU, so that the
CUDA path can be checked against it.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it; the product package
never does, and the oracle imports nothing from the product except the seeded
input generators (``paper_2408_03571_gb300.inputs``), which hold no solver
arithmetic.

Modules:
  problem        MP-1 / MP-2 finite-difference system (Section 2)
  decomposition  overlapping subdomains, R_i, D_i (Section 3)
  coarse         P_1 and B_2 coarse spaces, A_0 = R_0 A R_0^T (Section 4)
  schwarz        AS1, AS2 (Eq. 4), SAS2 (Eq. 5), SHS2 (Eq. 6)
  gmres          right-preconditioned GMRES / flexible GMRES (Section 5)
  adjoint        adjoint solve and d loss / d kappa (no counterpart in the paper)

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
printed values, invariants or library routines; see each module's docstring.
"""
from .problem import Problem, DIRICHLET, SOMMERFELD  # noqa: F401
from .decomposition import Decomposition  # noqa: F401
from .coarse import CoarseSpace, CoarseSolver, P1, B2, bspline2, basis_1d  # noqa: F401
from .schwarz import Schwarz, AS1, AS2, SAS2, SHS2, FP64, C64  # noqa: F401
from .gmres import gmres, givens  # noqa: F401
