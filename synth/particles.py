"""Seeded particle sets on a mesh: (face index, barycentric triple) plus tangent vectors."""
from __future__ import annotations

import numpy as np

from .meshes import Mesh, unwrapped_face_vertices


def face_areas(m: Mesh) -> np.ndarray:
    P = unwrapped_face_vertices(m)
    return 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)


def face_normals(m: Mesh) -> np.ndarray:
    P = unwrapped_face_vertices(m)
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def place_uniform(m: Mesh, n: int, seed: int, area_weighted: bool = True,
                  margin: float = 1e-6):
    """n points uniform on the surface (area weighted) or uniform over faces.

    Returns (face int32 (n,), bary float64 (n, 3)).  Barycentrics are drawn with
    the square-root rule and kept at least ``margin`` away from the face sides,
    so no particle starts exactly on an edge or a vertex.
    """
    rng = np.random.default_rng(seed)
    if area_weighted:
        a = face_areas(m)
        face = rng.choice(m.nf, size=n, p=a / a.sum())
    else:
        face = rng.integers(0, m.nf, size=n)
    u1 = rng.uniform(0.0, 1.0, n)
    u2 = rng.uniform(0.0, 1.0, n)
    r = np.sqrt(u1)
    bary = np.stack([1.0 - r, r * (1.0 - u2), r * u2], axis=1)
    bary = np.clip(bary, margin, None)
    bary /= bary.sum(axis=1, keepdims=True)
    return face.astype(np.int32), bary


def gaussian_tangent_velocities(m: Mesh, face: np.ndarray, kT: float, mass: float,
                                seed: int) -> np.ndarray:
    """World-frame velocities with N(0, kT/m) per tangent component.

    An isotropic 3D Gaussian projected on the face plane is an isotropic 2D
    Gaussian with the same per-component variance.
    """
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((face.shape[0], 3)) * np.sqrt(kT / mass)
    n = face_normals(m)[face]
    return v - np.sum(v * n, axis=1, keepdims=True) * n


def random_tangent_units(m: Mesh, face: np.ndarray, seed: int) -> np.ndarray:
    """Uniformly random unit tangent vectors (world frame) in each particle's face plane."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((face.shape[0], 3))
    n = face_normals(m)[face]
    v = v - np.sum(v * n, axis=1, keepdims=True) * n
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def world_positions(m: Mesh, face: np.ndarray, bary: np.ndarray) -> np.ndarray:
    """3D position of each particle (periodic meshes: wrapped into the period box)."""
    P = unwrapped_face_vertices(m)[face]
    x = np.einsum("nk,nkd->nd", bary, P)
    if m.period is not None:
        for ax, L in enumerate(m.period):
            x[:, ax] = np.mod(x[:, ax], L)
    return x
