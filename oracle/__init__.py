"""FP64 CPU oracle for the collocation Burton-Miller operator (Sec. 2, Eq.
eq_bm / eq_sum, discretised as in Sec. 5), its plane-wave right-hand side,
a dense LU and a matrix-free GMRES solve, and the closed forms that pin them
(Mie series and sphere eigenvalues).

TEST INFRASTRUCTURE.  Only tests/, the smoke check and the benchmark's CPU
baseline may import this package.  It shares no code with the CUDA library
(paper_1403_4747_gb300) and imports nothing from it.

Parity status per function:
  matvec / entry / assemble / rhs_plane_wave : pinned (kernels by finite
      differences, quadrature by exactness and brute force, operator by the
      sphere eigenvalues and the k -> 0 Gauss identity, solution by the Mie
      series, icosahedral symmetry).
  gmres / lu_solve                            : pinned (agree with each other
      and with the Mie series).
  mie_surface_field / sphere_eigenvalues      : pinned (mpmath evaluation,
      Rayleigh limit, mutual consistency).
"""
from .api import (load, geometry, kernels, integrate_triangle, self_hypersingular, entry,
                  is_near_pair, matvec, assemble, rhs_plane_wave, num_threads, gauss_legendre,
                  rule6, layer_rowsum)
from .solve import gmres, lu_solve
from .closed_forms import mie_surface_field, sphere_eigenvalue, legendre_on_mesh

__all__ = ["load", "geometry", "kernels", "integrate_triangle", "self_hypersingular", "entry",
           "is_near_pair", "matvec", "assemble", "rhs_plane_wave", "num_threads", "gauss_legendre",
           "rule6", "layer_rowsum", "gmres", "lu_solve", "mie_surface_field", "sphere_eigenvalue", "legendre_on_mesh"]
