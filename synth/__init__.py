"""Seeded synthetic inputs: triangulated surfaces and particle sets.

This package only *produces inputs* (vertex coordinates, face index triples,
particle faces / barycentric coordinates / initial velocities).  It contains
none of the geodesic, force or face-walk arithmetic; both the CPU oracle and
the CUDA library consume what it generates.
"""
from .meshes import (  # noqa: F401
    grid_plane, holed_plane, saddle_fan, cylinder_tube, cube, tetrahedron, octahedron, icosphere,
    torus, periodic_heightfield, bbox_diagonal, Mesh,
)
from .particles import place_uniform, gaussian_tangent_velocities, random_tangent_units  # noqa: F401
from .configs import make_config, CONFIG_NAMES  # noqa: F401
