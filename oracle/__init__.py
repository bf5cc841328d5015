"""Independent FP64 CPU oracle for the multibody axisymmetric Helmholtz BIE solver.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only `tests/`,
`__graft_entry__.smoke()` and the `cpu_baseline` / reference legs of `bench.py`
may import, call, link or execute anything here.  The CUDA library shares no code
with this package (no kernels, headers, helpers, tables or generators); the only
common input is the seeded generator module `workloads`, which holds no method
arithmetic.

What it computes (Hao, Martinsson, Young, "An efficient and highly accurate solver
for multi-body acoustic scattering problems involving rotationally symmetric
scatterers"):

  geometry.py  generating curves, Gauss-Legendre panels, tensor-product surface
               rule (Sec. 3.2), near-panel sets (Sec. 3.1)
  modal.py     modal kernels by brute-force azimuthal quadrature, per-mode Nystrom
               matrices with product integration on near panels, scattering
               matrices S_p = A~_p^{-1} (Sec. 3.2, Eqs. (seqBIE), (FAF), (singleinverse))
  operator.py  inter-body direct sum B (Sec. 3.3), block-diagonal inverse via the
               azimuthal DFT (Remark after Eq. (precond)), preconditioned apply,
               dense full matrix
  solvers.py   GMRES and a dense direct solve (Sec. 4)
  fields.py    plane waves, point sources, fields, far field, Mie series, sphere
               eigenvalues
  compress.py  the accelerated scheme (Sec. 5): proxy-sphere interpolative
               decomposition per shape, reduced system Eq. (ip6), density recovery
  liboracle.c  the plain-C double-precision loops behind the above

Every function is pinned by `tests/test_oracle_*.py` against closed forms,
library quadrature, invariants or brute force.
"""
from .geometry import NEAR_RHO, Rings, SurfaceNodes, gauss_legendre, near_panels, rings, surface_nodes
from .modal import modal_matrices, modal_system, scattering_matrices
from .operator import Problem
from .solvers import GmresResult, dense_solve, gmres
from . import fields

__all__ = ["NEAR_RHO", "Rings", "SurfaceNodes", "gauss_legendre", "near_panels", "rings",
           "surface_nodes", "modal_matrices", "modal_system", "scattering_matrices", "Problem",
           "GmresResult", "dense_solve", "gmres", "fields"]
