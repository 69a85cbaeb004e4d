"""Seeded synthetic inputs: tetrahedral meshes and nodal vorticity fields.

This package only builds inputs (node coordinates, tetrahedron connectivity,
nodal vorticity, sample indices) and the closed-form velocity of Hill's
spherical vortex that the tests and the benchmark compare against.  It holds
none of the velocity method's arithmetic, so both the CPU oracle and the CUDA
path can consume the same bytes without sharing any computation.
"""
from .mesh import kuhn_grid, jitter_interior, cube_to_ball, orient_positive, tet_volumes6
from .fields import (
    uniform_field,
    constant_plus_noise,
    gaussian_ring,
    two_rings,
    fourier_curl_field,
    gaussian_blob,
    hill_velocity,
    hill_vorticity,
)
from .configs import (
    Mesh,
    config1_plain,
    config2_ring,
    config3_fourier,
    config3_samples,
    config4_batch,
    config5_rings,
    ball_mesh,
)

__all__ = [
    "kuhn_grid", "jitter_interior", "cube_to_ball", "orient_positive", "tet_volumes6",
    "uniform_field", "constant_plus_noise", "gaussian_ring", "two_rings",
    "fourier_curl_field", "gaussian_blob", "hill_velocity", "hill_vorticity",
    "Mesh", "config1_plain", "config2_ring", "config3_fourier", "config3_samples",
    "config4_batch", "config5_rings", "ball_mesh",
]
