"""GB300-native geodesic molecular dynamics on triangulated surfaces.

The hot path (cutoff geodesic neighbours by window propagation, forces, the
face-walk integrators) runs in hand-written sm_103a CUDA behind the C ABI of
``include/css.h``; this package is its thin Python binding.
"""
from ._lib import (  # noqa: F401
    FP32, FP64, INT_ABP, INT_BD, INT_FIRE, INT_GD, INT_NVE, Launch, POT_GAUSSIAN, POT_HARMONIC, POT_WCA, Batch, Context,
    CssError, Integrator, Mesh, Particles, Potential, batch_create, batch_step, compute_forces,
    create, geodesic_neighbors, geodesic_paths, vhm_neighbors, integrate_step, trace_geodesics, load, mesh_upload, particles_get, particles_get_into, particles_set, particles_set_step, particles_update,
)
