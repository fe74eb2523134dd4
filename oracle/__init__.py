"""CPU oracle for the dense P1 stiffness matrix of the integral fractional Laplacian.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 restatement of
what the GPU path computes, written independently from the paper (Ainsworth &
Glusa, "Towards an efficient finite element method for the integral fractional
Laplacian on polygonal domains", Sections 2, 3, 5 and Appendix B).  Only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import it.  The product path never calls
it and shares no code, tables or constants with it.

Modules
-------
mesh      geometry, degrees of freedom, boundary facets, element-pair classes
rules     Gauss-Legendre rules and the collapsed (Duffy) triangle rule
assemble  element-pair assembly (Section 5, eqs. elementPair / elementPairBoundary)
exact     closed forms used as pins: C(d,s), ball solutions (Section 7),
          exact 1D matrix and exact 2D matrix through edge pairs
solve     Cholesky and Jacobi-preconditioned CG (Section 5)
heat      P1 mass matrix and implicit Euler steps of the fractional heat equation
          (Sections 2 and 5: systems (M + dt A^s) u = b)

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against a
closed form, a library routine on a special case, or brute force; none is
"parity unpinned".
"""
from . import mesh, rules, assemble, exact, solve, heat  # noqa: F401
from .mesh import OracleMesh  # noqa: F401
from .assemble import assemble_matrix, load_vector, QuadOrders  # noqa: F401
