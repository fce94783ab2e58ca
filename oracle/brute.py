"""Definitional geodesic distances on tiny meshes (TEST INFRASTRUCTURE ONLY).

A shortest path on a triangulated surface is a chain of straight segments, each
drawn in a planar unfolding of the faces it crosses, bending only at mesh
vertices (Sec. 2.2 of the paper: exact methods find the shortest straight path
inside the unfolded mesh).  This module computes that definition directly:

1. "direct" lengths: from a node (a surface point or a vertex) enumerate every
   sequence of faces a straight ray can cross, unfolding each next face into
   the plane of the first one and keeping the cone of ray directions that still
   passes through every crossed edge; a node lying inside the cone of a face of
   the sequence is reached by a straight segment of that length;
2. Dijkstra over the nodes {source, targets, all vertices} with those lengths.

Every vertex is allowed as a bend point, which only adds lengths of real paths,
so the minimum is the true distance.  A cone that has shrunk to a single ray
passes exactly through a vertex; such a path is the concatenation of two legs
through that vertex node and is not followed further.

It shares no code with the C oracle; it is slow (pure Python) and meant for
meshes of a few dozen faces.
"""
from __future__ import annotations

import heapq
import math
from typing import Dict, List, Tuple

import numpy as np

_TWO_PI = 2.0 * math.pi


def _wrap(a: float) -> float:
    """angle folded into (-pi, pi]"""
    a = math.fmod(a + math.pi, _TWO_PI)
    if a <= 0.0:
        a += _TWO_PI
    return a - math.pi


class BruteMesh:
    def __init__(self, mesh):
        self.V = np.asarray(mesh.verts, float)
        self.F = [tuple(int(x) for x in f) for f in np.asarray(mesh.faces)]
        self.period = mesh.period
        self.nf = len(self.F)
        self.nv = self.V.shape[0]
        nbr: Dict[Tuple[int, int], int] = {}
        for f, tri in enumerate(self.F):
            for k in range(3):
                nbr[(tri[k], tri[(k + 1) % 3])] = f
        # across[f][k]: face on the other side of edge (F[f][k], F[f][k+1]) or -1
        self.across = [[nbr.get((tri[(k + 1) % 3], tri[k]), -1) for k in range(3)]
                       for tri in self.F]
        self.vfaces: List[List[int]] = [[] for _ in range(self.nv)]
        for f, tri in enumerate(self.F):
            for v in tri:
                self.vfaces[v].append(f)
        self._len: Dict[Tuple[int, int], float] = {}
        self.lay = []
        self.axes = []
        for tri in self.F:
            a, b, c = tri
            e1 = self.evec(a, b)
            e2 = self.evec(a, c)
            L = float(np.linalg.norm(e1))
            x = e1 / L
            n = np.cross(e1, e2)
            n /= np.linalg.norm(n)
            y = np.cross(n, x)
            self.lay.append(((0.0, 0.0), (L, 0.0), (float(e2 @ x), float(e2 @ y))))
            self.axes.append((x, y))

    def evec(self, a, b):
        d = self.V[b] - self.V[a]
        if self.period is not None:
            for ax, L in enumerate(self.period):
                d[ax] -= L * round(d[ax] / L)
        return d

    def elen(self, a: int, b: int) -> float:
        key = (a, b) if a < b else (b, a)
        v = self._len.get(key)
        if v is None:
            v = float(np.linalg.norm(self.evec(a, b)))
            self._len[key] = v
        return v

    def third(self, f: int, a: int, b: int) -> int:
        for x in self.F[f]:
            if x != a and x != b:
                return x
        raise ValueError("degenerate face")

    def edge_index(self, f: int, a: int, b: int) -> int:
        tri = self.F[f]
        for j in range(3):
            p, q = tri[j], tri[(j + 1) % 3]
            if (p == a and q == b) or (p == b and q == a):
                return j
        raise ValueError("edge not in face")


def _place_apex(A, B, la, lb, other):
    """third triangle vertex on segment AB with side lengths la (to A), lb (to B), placed
    on the side of line AB opposite to the point 'other'."""
    dx, dy = B[0] - A[0], B[1] - A[1]
    L = math.hypot(dx, dy)
    ux, uy = dx / L, dy / L
    x = (la * la - lb * lb + L * L) / (2.0 * L)
    y = math.sqrt(max(la * la - x * x, 0.0))
    side = dx * (other[1] - A[1]) - dy * (other[0] - A[0])
    nx, ny = (-uy, ux) if side <= 0 else (uy, -ux)
    return (A[0] + x * ux + y * nx, A[1] + x * uy + y * ny)


def _rel(c: float, px: float, py: float) -> float:
    return c + _wrap(math.atan2(py, px) - c)


def direct_lengths(bm: BruteMesh, start, dmax: float, targets, min_width: float = 1e-9):
    """Straight-segment lengths from a start node to every node it sees directly.

    start: ("pt", face, bary) or ("v", vertex).  targets: list of (face, bary).
    Returns {("v", i) | ("t", i): (length, direction (dx, dy))}; for a point start the
    direction is expressed in the layout of the start face.
    """
    out: Dict[tuple, Tuple[float, Tuple[float, float]]] = {}
    tgt_by_face: Dict[int, List[int]] = {}
    for ti, (tf, _) in enumerate(targets):
        tgt_by_face.setdefault(int(tf), []).append(ti)

    def record(key, dx, dy):
        L = math.hypot(dx, dy)
        if L > 0.0 and (key not in out or L < out[key][0]):
            out[key] = (L, (dx, dy))

    def visit(g, P, A, lo, hi):
        c = 0.5 * (lo + hi)
        for v in bm.F[g]:
            dx, dy = P[v][0] - A[0], P[v][1] - A[1]
            if dx == 0.0 and dy == 0.0:
                continue
            a = _rel(c, dx, dy)
            if lo - 1e-12 <= a <= hi + 1e-12:
                record(("v", v), dx, dy)
        for ti in tgt_by_face.get(g, ()):
            tb = targets[ti][1]
            a0, b0, c0 = bm.F[g]
            X = (tb[0] * P[a0][0] + tb[1] * P[b0][0] + tb[2] * P[c0][0],
                 tb[0] * P[a0][1] + tb[1] * P[b0][1] + tb[2] * P[c0][1])
            dx, dy = X[0] - A[0], X[1] - A[1]
            if dx == 0.0 and dy == 0.0:
                continue
            a = _rel(c, dx, dy)
            if lo - 1e-12 <= a <= hi + 1e-12:
                record(("t", ti), dx, dy)

    def walk(g, P, A, lo, hi, entry, depth):
        """cross every edge of face g but the entry edge, clipping the cone [lo, hi]."""
        if depth > 400:
            return
        c = 0.5 * (lo + hi)
        tri = bm.F[g]
        for k in range(3):
            if k == entry:
                continue
            h = bm.across[g][k]
            if h < 0:
                continue
            a, b = tri[k], tri[(k + 1) % 3]
            Pa, Pb = P[a], P[b]
            ea = _rel(c, Pa[0] - A[0], Pa[1] - A[1])
            eb = _rel(c, Pb[0] - A[0], Pb[1] - A[1])
            if ea > eb:
                ea, eb = eb, ea
            if eb - ea >= math.pi:              # segment behind the apex
                continue
            nlo, nhi = max(lo, ea), min(hi, eb)
            if nhi - nlo <= min_width:          # empty, or a single ray through a vertex
                continue
            ex, ey = Pb[0] - Pa[0], Pb[1] - Pa[1]
            t = ((A[0] - Pa[0]) * ex + (A[1] - Pa[1]) * ey) / (ex * ex + ey * ey)
            t = 0.0 if t < 0.0 else (1.0 if t > 1.0 else t)
            if math.hypot(Pa[0] + t * ex - A[0], Pa[1] + t * ey - A[1]) > dmax:
                continue
            cc = bm.third(h, a, b)
            Pc = _place_apex(Pa, Pb, bm.elen(a, cc), bm.elen(b, cc), P[bm.third(g, a, b)])
            Q = {a: Pa, b: Pb, cc: Pc}
            visit(h, Q, A, nlo, nhi)
            walk(h, Q, A, nlo, nhi, bm.edge_index(h, a, b), depth + 1)

    def fan(f, P, A, a, b, opp_k):
        """start a cone from apex A (inside or at a corner of face f) through edge (a, b)."""
        h = bm.across[f][opp_k]
        if h < 0:
            return
        ta = math.atan2(P[a][1] - A[1], P[a][0] - A[0])
        tb = ta + _wrap(math.atan2(P[b][1] - A[1], P[b][0] - A[0]) - ta)
        lo, hi = min(ta, tb), max(ta, tb)
        cc = bm.third(h, a, b)
        Pc = _place_apex(P[a], P[b], bm.elen(a, cc), bm.elen(b, cc), P[bm.third(f, a, b)])
        Q = {a: P[a], b: P[b], cc: Pc}
        visit(h, Q, A, lo, hi)
        walk(h, Q, A, lo, hi, bm.edge_index(h, a, b), 1)

    if start[0] == "pt":
        f0, b0 = int(start[1]), start[2]
        Pl = bm.lay[f0]
        P = {bm.F[f0][k]: Pl[k] for k in range(3)}
        A = (b0[0] * Pl[0][0] + b0[1] * Pl[1][0] + b0[2] * Pl[2][0],
             b0[0] * Pl[0][1] + b0[1] * Pl[1][1] + b0[2] * Pl[2][1])
        for v in bm.F[f0]:
            record(("v", v), P[v][0] - A[0], P[v][1] - A[1])
        for ti in tgt_by_face.get(f0, ()):
            tb = targets[ti][1]
            X = (tb[0] * Pl[0][0] + tb[1] * Pl[1][0] + tb[2] * Pl[2][0],
                 tb[0] * Pl[0][1] + tb[1] * Pl[1][1] + tb[2] * Pl[2][1])
            record(("t", ti), X[0] - A[0], X[1] - A[1])
        for k in range(3):
            fan(f0, P, A, bm.F[f0][k], bm.F[f0][(k + 1) % 3], k)
    else:
        v0 = int(start[1])
        for f in bm.vfaces[v0]:
            Pl = bm.lay[f]
            tri = bm.F[f]
            P = {tri[k]: Pl[k] for k in range(3)}
            A = P[v0]
            k0 = tri.index(v0)
            a, b = tri[(k0 + 1) % 3], tri[(k0 + 2) % 3]
            record(("v", a), P[a][0] - A[0], P[a][1] - A[1])
            record(("v", b), P[b][0] - A[0], P[b][1] - A[1])
            for ti in tgt_by_face.get(f, ()):
                tb = targets[ti][1]
                X = (tb[0] * Pl[0][0] + tb[1] * Pl[1][0] + tb[2] * Pl[2][0],
                     tb[0] * Pl[0][1] + tb[1] * Pl[1][1] + tb[2] * Pl[2][1])
                record(("t", ti), X[0] - A[0], X[1] - A[1])
            fan(f, P, A, a, b, (k0 + 1) % 3)
        out.pop(("v", v0), None)
    return out


def geodesics(mesh, f0: int, b0, targets, dmax: float):
    """(distances, tangent_world) from point (f0, b0) to each target (face, bary).

    dmax bounds the length of every straight leg that is searched.
    """
    bm = BruteMesh(mesh)
    src = direct_lengths(bm, ("pt", f0, tuple(float(x) for x in b0)), dmax, targets)
    vdir = {}
    dist: Dict[tuple, float] = {}
    first: Dict[tuple, Tuple[float, float]] = {}
    pq = [(L, key, d) for key, (L, d) in src.items()]
    heapq.heapify(pq)
    while pq:
        L, key, d = heapq.heappop(pq)
        if key in dist:
            continue
        dist[key] = L
        first[key] = d
        if key[0] == "v":
            v = key[1]
            if v not in vdir:
                vdir[v] = direct_lengths(bm, ("v", v), dmax, targets)
            for k2, (L2, _) in vdir[v].items():
                if k2 not in dist:
                    heapq.heappush(pq, (L + L2, k2, d))
    x, y = bm.axes[int(f0)]
    D = np.full(len(targets), math.inf)
    T = np.zeros((len(targets), 3))
    for i in range(len(targets)):
        if ("t", i) in dist:
            D[i] = dist[("t", i)]
            dx, dy = first[("t", i)]
            n = math.hypot(dx, dy)
            T[i] = (dx * x + dy * y) / n
    return D, T
