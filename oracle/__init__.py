"""FP64 CPU oracle for the NanoBTE hot path -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct reference the CUDA path is
checked against.  It is used only by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline / reference legs of ``bench.py``; the library and its
Python binding never import, call or execute anything here, and this package
imports nothing from them (only the seeded input generators in ``workloads``
are shared, and they hold none of the method's arithmetic).

What it follows (equation numbers are the paper's, counted in order of
appearance in Sec. II "Methods"):

* Eq. (4)  steady per-mode BTE  ``v s_i . grad e + (e - e0)/tau = S``,
  discretised with first-order upwind finite volumes; each (band, direction)
  task is the sparse system ``A = I/tau + v K_i`` of Eq. (13), factorised once
  (``scipy.sparse.linalg.splu``) and reused every iteration.
* Eq. (5)  lattice (pseudo-)temperature from the collision moment.
* Eq. (7)  heat flux moment; energy temperature ``T = sum w e / C_tot``.
* Eq. (11) equilibrium ``e0 = C T / W``.
* Eqs. (8)-(10) synthetic diffusion correction, solved with a sparse LU of the
  cell Laplacian (the paper's "cached macroscopic LU").
* Sec. III B: heat source as an equilibrium source, uniform over directions,
  split over bands by heat capacity.
* Walls (thermalizing / diffuse / specular / partially specular) with the
  reflected values taken from the previous iteration.
* Optional second-order upwind face values (``order=2``): the gradient
  operators the paper builds once from the mesh (Sec. II), read as a linear
  reconstruction from the upwind cell with a least-squares gradient of the
  previous iteration's distribution, as a right-hand-side correction of the
  same factorised system.

Points the paper leaves open are read as follows, and each function below
names the reading it uses: first-order step upwind by default (second order
on interior faces only, and only from cells with at least dim + 1 face
neighbours, when asked for); wall values lagged one
outer iteration; the synthetic update in its DSA form (the diffusion term at
the kinetic temperature, Eqs. (8)-(10)), with the correction's equilibrium
part added to the lagged wall values; a TPFA cell Laplacian with the upwind
scheme's numerical diffusivity added to kappa; convergence measured as
max|dT'| / max|T'|.

Parity status: the transport/moment/wall arithmetic is pinned by the tests in
``tests/test_oracle_pins.py`` (closed forms, invariants, brute-force dense
solves), the second-order reconstruction by ``tests/test_oracle_order2.py``
(linear exactness, the per-cell energy identity, dense solves of the
second-order system, the measured order of accuracy).  The synthetic *iteration path* (how fast it converges) is not pinned
beyond "reaches the same fixed point as the sequential scheme"; the fixed point
itself is.
"""
from .geometry import Geometry, build_geometry
from .bte import OracleSolver, quadrature_moments

__all__ = ["Geometry", "build_geometry", "OracleSolver", "quadrature_moments"]
