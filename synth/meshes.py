"""Procedural triangulated surfaces (vertices V x 3 float64, faces F x 3 int32).

All faces are oriented counter-clockwise when seen from the side the outward
normal points to, so every interior edge appears once as (a, b) and once as
(b, a).  Periodic meshes carry ``period = (Lx, Ly)``: their connectivity wraps
in x and y and vertex x/y coordinates lie in [0, Lx) x [0, Ly).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np


@dataclass
class Mesh:
    verts: np.ndarray                 # (V, 3) float64
    faces: np.ndarray                 # (F, 3) int32
    period: Optional[Tuple[float, float]] = None
    name: str = "mesh"
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nf(self) -> int:
        return int(self.faces.shape[0])


def _mk(verts, faces, period=None, name="mesh", **meta) -> Mesh:
    return Mesh(np.ascontiguousarray(verts, dtype=np.float64),
                np.ascontiguousarray(faces, dtype=np.int32), period, name, dict(meta))


def grid_plane(nx: int = 21, ny: int = 21, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
               alternate: bool = False) -> Mesh:
    """Open flat rectangle, nx x ny vertex grid, every quad split in 2 (normal +z)."""
    xs = np.linspace(x0, x1, nx)
    ys = np.linspace(y0, y1, ny)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    verts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    faces = []
    for j in range(ny - 1):
        for i in range(nx - 1):
            a = j * nx + i
            b = a + 1
            c = a + nx
            d = c + 1
            if alternate and (i + j) % 2:
                faces += [(a, b, c), (b, d, c)]
            else:
                faces += [(a, b, d), (a, d, c)]
    return _mk(verts, faces, name=f"plane{nx}x{ny}")


def holed_plane(n: int = 21, hole=(0.4, 0.6, 0.4, 0.6)) -> Mesh:
    """The open flat unit square of ``grid_plane(n, n)`` with the grid cells inside the
    rectangle hole = (x0, x1, y0, y1) removed (a square hole whose sides lie on grid
    lines), unused vertices dropped.  Shortest paths on it wrap around the hole's corners."""
    g = grid_plane(n, n)
    x0, x1, y0, y1 = hole
    c = g.verts[g.faces].mean(axis=1)
    keep = ~((c[:, 0] > x0) & (c[:, 0] < x1) & (c[:, 1] > y0) & (c[:, 1] < y1))
    faces = g.faces[keep]
    used = np.unique(faces)
    remap = -np.ones(g.nv, np.int64)
    remap[used] = np.arange(used.size)
    return _mk(g.verts[used], remap[faces], name=f"holed_plane{n}")


def saddle_fan(n_sectors: int = 8, subdiv: int = 4) -> Mesh:
    """Open fan of n_sectors (even) equilateral triangles of unit side around one apex, each
    split flat into subdiv^2 triangles.  The rim vertices alternate above and below the
    apex's plane so that consecutive ones are one unit apart: the apex's total angle is
    n_sectors * pi/3 (8 sectors: 8 pi/3 > 2 pi, a saddle vertex).  meta["rim"] holds the
    rim directions (unit vectors from the apex)."""
    assert n_sectors % 2 == 0 and n_sectors >= 6
    dlon = 2 * np.pi / n_sectors
    # latitude b with chord 1 between (b, 0) and (-b, dlon): cos 60deg = cos^2 b cos dlon - sin^2 b
    c2 = 1.5 / (1.0 + np.cos(dlon))
    b = np.arccos(np.sqrt(c2))
    rim = np.array([[np.cos(b) * np.cos(k * dlon), np.cos(b) * np.sin(k * dlon), (1 if k % 2 == 0 else -1) * np.sin(b)]
                    for k in range(n_sectors)])
    verts, faces, index = [], [], {}

    def vid(s_, i, j):
        # point apex + (i/subdiv) u_s + (j/subdiv) u_{s+1}, i + j <= subdiv; shared across sectors
        if i + j == 0:
            key = ("apex",)
        elif j == 0:
            key = ("ray", s_ % n_sectors, i)
        elif i == 0:
            key = ("ray", (s_ + 1) % n_sectors, j)
        else:
            key = ("in", s_ % n_sectors, i, j)
        if key not in index:
            index[key] = len(verts)
            verts.append((i * rim[s_ % n_sectors] + j * rim[(s_ + 1) % n_sectors]) / subdiv)
        return index[key]

    for s_ in range(n_sectors):
        for i in range(subdiv):
            for j in range(subdiv - i):
                faces.append((vid(s_, i, j), vid(s_, i + 1, j), vid(s_, i, j + 1)))
                if i + j + 2 <= subdiv:
                    faces.append((vid(s_, i + 1, j), vid(s_, i + 1, j + 1), vid(s_, i, j + 1)))
    return _mk(np.array(verts), faces, name=f"saddle_fan{n_sectors}", rim=rim)


def cylinder_tube(n_around: int = 12, n_along: int = 6, radius: float = 1.0,
                  height: float = 2.0) -> Mesh:
    """Open prism tube (n_around-gon cross-section) of the given height, outward normals."""
    verts = []
    for k in range(n_along + 1):
        z = height * k / n_along
        for i in range(n_around):
            a = 2.0 * np.pi * i / n_around
            verts.append((radius * np.cos(a), radius * np.sin(a), z))
    faces = []
    for k in range(n_along):
        for i in range(n_around):
            a = k * n_around + i
            b = k * n_around + (i + 1) % n_around
            c = a + n_around
            d = b + n_around
            faces += [(a, b, d), (a, d, c)]
    return _mk(verts, faces, name=f"tube{n_around}x{n_along}",
               radius=radius, height=height, n_around=n_around)


def _weld(verts, faces, decimals=12):
    key = np.round(np.asarray(verts), decimals)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.ravel()
    # keep the first original coordinates of each welded vertex
    out = np.zeros_like(uniq)
    out[inv] = np.asarray(verts)
    return out, inv[np.asarray(faces)]


def cube(n: int = 1, size: float = 1.0) -> Mesh:
    """Surface of the cube [0,size]^3, each side an n x n grid of quads split in 2."""
    verts, faces = [], []
    # (origin, u axis, v axis) with u x v = outward normal
    sides = [
        ((0, 0, 0), (0, 1, 0), (1, 0, 0)),  # z = 0, normal -z
        ((0, 0, 1), (1, 0, 0), (0, 1, 0)),  # z = 1, normal +z
        ((0, 0, 0), (1, 0, 0), (0, 0, 1)),  # y = 0, normal -y
        ((0, 1, 0), (0, 0, 1), (1, 0, 0)),  # y = 1, normal +y
        ((0, 0, 0), (0, 0, 1), (0, 1, 0)),  # x = 0, normal -x
        ((1, 0, 0), (0, 1, 0), (0, 0, 1)),  # x = 1, normal +x
    ]
    for o, u, v in sides:
        o, u, v = (np.array(t, float) for t in (o, u, v))
        base = len(verts)
        for j in range(n + 1):
            for i in range(n + 1):
                verts.append(size * (o + u * i / n + v * j / n))
        for j in range(n):
            for i in range(n):
                a = base + j * (n + 1) + i
                b = a + 1
                c = a + (n + 1)
                d = c + 1
                faces += [(a, b, d), (a, d, c)]
    V, Fc = _weld(np.array(verts), np.array(faces))
    return _mk(V, Fc, name=f"cube{n}", size=size)


def tetrahedron(scale: float = 1.0) -> Mesh:
    v = scale * np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float)
    f = [(0, 1, 2), (0, 3, 1), (0, 2, 3), (1, 3, 2)]
    return _fix_outward(_mk(v, f, name="tetra"))


def octahedron(scale: float = 1.0) -> Mesh:
    v = scale * np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    f = [(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4), (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)]
    return _fix_outward(_mk(v, f, name="octa"))


def _fix_outward(m: Mesh) -> Mesh:
    """Flip faces of a star-shaped closed mesh so normals point away from its centroid."""
    c = m.verts.mean(axis=0)
    F = m.faces.copy()
    for k, (a, b, d) in enumerate(F):
        n = np.cross(m.verts[b] - m.verts[a], m.verts[d] - m.verts[a])
        if np.dot(n, m.verts[a] + m.verts[b] + m.verts[d] - 3 * c) < 0:
            F[k] = (a, d, b)
    m.faces = F.astype(np.int32)
    return m


_ICO_F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
          (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
          (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
          (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]


def icosphere(level: int = 5, radius: float = 1.0, noise: float = 0.0,
              seed: int = 0) -> Mesh:
    """Subdivided icosahedron on a sphere; optional radial displacement noise*N(0,1)."""
    t = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    V = np.array(v, float)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array(_ICO_F, np.int64)
    for _ in range(level):
        nv = V.shape[0]
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        ue, inv = np.unique(e, axis=0, return_inverse=True)
        inv = inv.ravel()
        mid = V[ue[:, 0]] + V[ue[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        V = np.concatenate([V, mid], axis=0)
        nfc = F.shape[0]
        m01 = nv + inv[:nfc]
        m12 = nv + inv[nfc:2 * nfc]
        m20 = nv + inv[2 * nfc:]
        a, b, c = F[:, 0], F[:, 1], F[:, 2]
        F = np.concatenate([np.stack([a, m01, m20], 1), np.stack([b, m12, m01], 1),
                            np.stack([c, m20, m12], 1), np.stack([m01, m12, m20], 1)], 0)
    V = V * radius
    if noise > 0.0:
        rng = np.random.default_rng(seed)
        g = rng.standard_normal(V.shape[0])
        V = V * ((radius + noise * g) / radius)[:, None]
    m = _mk(V, F, name=f"ico{level}", radius=radius, level=level, noise=noise)
    # orientation of the base icosahedron list is consistent; make it outward
    a, b, c = m.verts[m.faces[0]]
    if np.dot(np.cross(b - a, c - a), a + b + c) < 0:
        m.faces = m.faces[:, [0, 2, 1]].copy()
    return m


def torus(R: float = 3.0, r: float = 1.0, n_u: int = 48, n_v: int = 24) -> Mesh:
    """Ring torus, major radius R, minor radius r, n_u x n_v quads split in 2."""
    u = 2 * np.pi * np.arange(n_u) / n_u
    v = 2 * np.pi * np.arange(n_v) / n_v
    U, Vv = np.meshgrid(u, v, indexing="ij")
    X = (R + r * np.cos(Vv)) * np.cos(U)
    Y = (R + r * np.cos(Vv)) * np.sin(U)
    Z = r * np.sin(Vv)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    idx = lambda i, j: (i % n_u) * n_v + (j % n_v)
    faces = []
    for i in range(n_u):
        for j in range(n_v):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i, j + 1), idx(i + 1, j + 1)
            faces += [(a, b, d), (a, d, c)]
    return _mk(verts, faces, name=f"torus{n_u}x{n_v}", R=R, r=r)


def periodic_heightfield(n: int = 256, n_gauss: int = 32, seed: int = 3,
                         A=(0.05, 0.3), w=(0.05, 0.2)) -> Mesh:
    """z = sum_k A_k exp(-|x-c_k|^2 / (2 w_k^2)) on the unit periodic square.

    The Gaussians are summed over their 3x3 periodic images so z is smooth and
    periodic; the grid is n x n with wrapped connectivity, period (1, 1).
    """
    rng = np.random.default_rng(seed)
    Ak = rng.uniform(A[0], A[1], n_gauss)
    wk = rng.uniform(w[0], w[1], n_gauss)
    ck = rng.uniform(0.0, 1.0, (n_gauss, 2))
    xs = np.arange(n) / n
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    Z = np.zeros_like(X)
    for k in range(n_gauss):
        for sx in (-1, 0, 1):
            for sy in (-1, 0, 1):
                dx = X - ck[k, 0] - sx
                dy = Y - ck[k, 1] - sy
                Z += Ak[k] * np.exp(-(dx * dx + dy * dy) / (2 * wk[k] ** 2))
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    idx = lambda i, j: (j % n) * n + (i % n)
    faces = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i, j + 1), idx(i + 1, j + 1)
            faces += [(a, b, d), (a, d, c)]
    return _mk(verts, faces, period=(1.0, 1.0), name=f"hfield{n}",
               A=Ak, w=wk, c=ck)


def unwrapped_face_vertices(m: Mesh) -> np.ndarray:
    """(F, 3, 3) vertex coordinates of every face, periodic images unwrapped around vertex 0."""
    P = m.verts[m.faces]
    if m.period is not None:
        for ax, L in enumerate(m.period):
            for k in (1, 2):
                d = P[:, k, ax] - P[:, 0, ax]
                P[:, k, ax] -= L * np.round(d / L)
    return P


def bbox_diagonal(m: Mesh) -> float:
    """Length used as the 'mesh diameter' scale for relative FP32 error bars."""
    ext = m.verts.max(axis=0) - m.verts.min(axis=0)
    if m.period is not None:
        ext[0], ext[1] = m.period
    return float(np.linalg.norm(ext))
