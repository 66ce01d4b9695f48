"""FP64 CPU oracle of the third-order unstructured WENO scheme (arXiv 1712.08317).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
reference legs use it.  It shares no code with the CUDA library; the two meet
only through the seeded inputs of the `synthetic` package.

Plain numpy, float64 throughout, vectorised across cells but with every
cell-local step written in the paper's order:

  mesh.py           Section 2: cells, faces, outward normals, edge Gauss points
                    (Eq. 5); Sections 3.1/3.2: the general stencil with its
                    E_j flags and replacement rules.
  reconstruction.py Sections 3.1-3.3: the quadratic P^2 by least squares
                    (Eqs. 9-12), candidate linear polynomials, the linear
                    weight system B gamma = eta (Eq. 15) and the optimisation
                    of large weights (weighting parameters d_j).
  weno.py           Section 3.4: splitting of negative weights, the new
                    smoothness indicator, nonlinear weights and the Gauss-point
                    values.
  flux.py           Eq. 6 rotation + HLLC (Toro) for Euler; exact upwind for
                    scalar advection.
  scheme.py         Eq. 4 residual, SSP-RK3 (Section 4), CFL time step.

Readings of points the paper leaves open are fixed in one place
(`Params` and the docstrings) and listed with the design notes.

Parity pins: every function here is pinned by tests/test_oracle_*.py against
closed forms, invariants, textbook special cases or brute force, except the
exact digits of the nonlinear weights at a given point (no worked example in
the paper): parity unpinned for those digits beyond the invariants
(free-stream preservation, exact linear reproduction, reduction to the
linear scheme when beta -> 0).
"""
from .mesh import OracleMesh
from .reconstruction import Params, precompute
from .scheme import OracleSolver, NonPhysicalState

__all__ = ["OracleMesh", "Params", "precompute", "OracleSolver", "NonPhysicalState"]
