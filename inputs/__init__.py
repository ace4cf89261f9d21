"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds only input generation: surface meshes (icospheres and the
ellipsoid mapped from them), incidence directions and seeded random complex
vectors.  It contains none of the boundary-element arithmetic, so both the
oracle and the GPU library can take their inputs from here without sharing
any of the method's code.

The paper's own meshes (sphere families of Sec. 5, the Su-27 and submarine of
Sec. 5.3) are not available; the icosphere family stands in for the sphere
meshes of Table tab_usphpls and the plane-wave sphere of Sec. 5.3.
"""
from .meshes import (icosphere, octasphere, ellipsoid_from_icosphere, fibonacci_directions,
                     complex_normal, icosahedral_rotations, mesh_for_config, multi_mesh_set)

__all__ = ["icosphere", "octasphere", "ellipsoid_from_icosphere", "fibonacci_directions",
           "complex_normal", "icosahedral_rotations", "mesh_for_config", "multi_mesh_set"]
