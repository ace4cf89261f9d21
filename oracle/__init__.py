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
  rhs_layers_matvec / rhs_layers_assemble /
  self_single_layer                           : pinned (self integral by a
      Duffy-transformed brute force and the equilateral closed form, operator
      by the sphere eigenvalues beta_n and the k -> 0 potential of a uniform
      layer, pulsating-sphere solution converging to 1/(1 - ik)).
"""
from .api import (load, geometry, kernels, integrate_triangle, self_hypersingular, entry,
                  is_near_pair, matvec, assemble, rhs_plane_wave, num_threads, gauss_legendre,
                  rule6, layer_rowsum, rhs_layers_matvec, rhs_layers_assemble, rhs_layers_entry,
                  self_single_layer, rhs_point_source, scattered_field, far_field)
from .solve import gmres, lu_solve
from .closed_forms import (mie_surface_field, sphere_eigenvalue, legendre_on_mesh, sphere_rhs_eigenvalue,
                           pulsating_sphere_potential, point_source_surface_field, mie_scattered_field,
                           mie_far_field)

__all__ = ["load", "geometry", "kernels", "integrate_triangle", "self_hypersingular", "entry",
           "is_near_pair", "matvec", "assemble", "rhs_plane_wave", "num_threads", "gauss_legendre",
           "rule6", "layer_rowsum", "gmres", "lu_solve", "mie_surface_field", "sphere_eigenvalue", "legendre_on_mesh",
           "rhs_layers_matvec", "rhs_layers_assemble", "rhs_layers_entry", "self_single_layer",
           "sphere_rhs_eigenvalue", "pulsating_sphere_potential", "rhs_point_source",
           "point_source_surface_field", "scattered_field", "far_field", "mie_scattered_field", "mie_far_field"]
