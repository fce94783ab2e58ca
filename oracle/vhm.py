"""Oracle of the approximate distance solver: heat-method distances with vector-heat
transport for the initial tangents.  TEST INFRASTRUCTURE: only the tests, the smoke check
and the benchmark's CPU-baseline leg use it; the library never does.

The paper names the vector heat method (Sharp, Soliman & Crane 2019) as the approximate,
faster alternative to exact window propagation, with O(h) distance error on a mesh of
spacing h (Sec. 2.2, and again as future work in Sec. 5).  What is computed here, for a
source point q in face f0 with barycentrics b, on the triangle mesh as it is (intrinsic
edge lengths; minimum-image edges on periodic meshes), in FP64 with direct sparse solves:

  1. operators (Crane et al. 2013; Sharp et al. 2019):
       L   cotan Laplacian, positive semi-definite: L_ij = -w_ij, L_ii = sum_j w_ij,
           w_ij = (cot a + cot b) / 2 over the corners opposite edge ij;
       M   lumped mass, a third of the incident face areas;
       vertex tangent frames: the corners around vertex v in counter-clockwise order from
           a reference corner, the angle phi of each corner's outgoing edge being the
           summed corner angles scaled by s_v = 2 pi / Theta_v (pi / Theta_v on the
           boundary), so every vertex's tangent directions close up to a full turn;
       a face-plane direction at corner k of face f with layout angle beta becomes the
           vertex-frame angle phi(f, k) + s_v * wrap(beta - gamma(f, k)), gamma the layout
           angle of the corner's outgoing edge, wrap() into (-pi, pi];
       Lc  connection Laplacian (Hermitian PSD): Lc_ii = sum_j w_ij, Lc_ij = -w_ij r_ji,
           r_ji = exp(i (phi_ij + pi - phi_ji)) carrying a vector at j into i's frame
           (phi_ij: angle at i of the edge towards j);
       t   = t_factor * (mean edge length)^2.
  2. scalar heat, one backward-Euler step: (M + t L) u = u0, u0 = b on f0's corners;
  3. vector heat, one backward-Euler step: (M + t Lc) Y = Y0, Y0 = b_k times the unit
     x-axis of f0's layout carried into corner k's frame; H = Y / |Y| (the transported
     reference direction);
  4. X_f = -grad u / |grad u| per face (unit, pointing away from the source; 0 where the
     gradient vanishes, i.e. where u underflowed: beyond about 700 sqrt(t) from the source);
  5. Poisson: L phi = -div X with (div X)_i = 1/2 sum over faces at i of
     cot(theta_1) (e_1 . X) + cot(theta_2) (e_2 . X) (e_1, e_2 the face's edges from i,
     theta_1, theta_2 the angles opposite them), phi fixed by phi(q) = 0 (q interpolated);
  6. per target y in face g with barycentrics c: distance d = sum_k c_k phi(v_k);
     the direction away from the source at y is G_g = grad phi on g (the computed distance
     field's own gradient; X only feeds the Poisson right-hand side);
     angle theta = arg sum_k c_k exp(i psi_k) conj(H_k), psi_k the vertex-frame angle of
     G_g at corner k; the tangent at q is f0's layout x-axis turned by theta (world frame).

Parity unpinned: no.  Pins (tests/test_oracle_vhm.py): the cotan Laplacian annihilates
constants everywhere and linear functions at interior vertices of a flat mesh; the mass
sums to the area; a globally parallel field on a flat periodic patch lies in the kernel of
the connection Laplacian (a wrong transport phase fails); there the transported reference
is the constant field; distances and tangents converge to the great-circle ones on the
unit sphere at first order in h and to the Euclidean ones on a flat periodic patch; on a
noisy sphere they stay within a few percent of the exact polyhedral distances.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _wrap(a):
    """Angles into (-pi, pi]."""
    return a - 2.0 * math.pi * np.ceil((a - math.pi) / (2.0 * math.pi))


class VhmMesh:
    def __init__(self, mesh, t_factor: float = 1.0):
        X = np.asarray(mesh.verts, np.float64)
        F = np.asarray(mesh.faces, np.int64)
        self.mesh, self.X, self.F = mesh, X, F
        nv, nf = X.shape[0], F.shape[0]
        self.nv, self.nf = nv, nf
        per = mesh.period

        def edge(a, b):
            d = X[b] - X[a]
            if per is not None:
                d[:, 0] -= per[0] * np.round(d[:, 0] / per[0])
                d[:, 1] -= per[1] * np.round(d[:, 1] / per[1])
            return d
        # corner k of face f: edge lengths of the three sides, planar layout (corner 0 at the
        # origin, corner 1 on +x, corner 2 above)
        e01 = edge(F[:, 0], F[:, 1])
        e02 = edge(F[:, 0], F[:, 2])
        l01 = np.linalg.norm(e01, axis=1)
        l02 = np.linalg.norm(e02, axis=1)
        l12 = np.linalg.norm(edge(F[:, 1], F[:, 2]), axis=1)
        x2 = (l01 ** 2 + l02 ** 2 - l12 ** 2) / (2.0 * l01)
        y2 = np.sqrt(np.maximum(l02 ** 2 - x2 ** 2, 0.0))
        P = np.zeros((nf, 3, 2))
        P[:, 1, 0] = l01
        P[:, 2, 0] = x2
        P[:, 2, 1] = y2
        self.P = P
        # world frame of each layout: E1 along corner 0 -> 1, E2 in the face plane
        E1 = e01 / l01[:, None]
        nrm = np.cross(e01, e02)
        nrm /= np.linalg.norm(nrm, axis=1)[:, None]
        self.E1, self.E2 = E1, np.cross(nrm, E1)
        self.area = 0.5 * l01 * y2
        # corner angles and the layout angle of each corner's outgoing edge (k -> k+1)
        ang = np.zeros((nf, 3))
        gam = np.zeros((nf, 3))
        for k in range(3):
            a, b, c = P[:, k], P[:, (k + 1) % 3], P[:, (k + 2) % 3]
            u, w = b - a, c - a
            ang[:, k] = np.arctan2(u[:, 0] * w[:, 1] - u[:, 1] * w[:, 0], u[:, 0] * w[:, 0] + u[:, 1] * w[:, 1])
            gam[:, k] = np.arctan2(u[:, 1], u[:, 0])
        self.ang, self.gam = ang, gam
        cot = 1.0 / np.tan(ang)
        # cotan Laplacian and lumped mass
        rows, cols, vals = [], [], []
        for k in range(3):
            i, j = F[:, (k + 1) % 3], F[:, (k + 2) % 3]
            w = 0.5 * cot[:, k]
            rows += [i, j, i, j]
            cols += [j, i, i, j]
            vals += [-w, -w, w, w]
        self.L = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nv, nv))
        self.M = sp.diags(np.bincount(F.ravel(), weights=np.repeat(self.area / 3.0, 3), minlength=nv))
        self.cot = cot
        # half-edge twins (h = 3 f + k runs from corner k to k + 1)
        key = {}
        for f in range(nf):
            for k in range(3):
                key[(int(F[f, k]), int(F[f, (k + 1) % 3]))] = 3 * f + k
        twin = np.full(3 * nf, -1, np.int64)
        for (a, b), h in key.items():
            twin[h] = key.get((b, a), -1)
        self.twin = twin
        # vertex frames: corners of each vertex walked counter-clockwise
        theta = np.bincount(F.ravel(), weights=ang.ravel(), minlength=nv)
        corners = [[] for _ in range(nv)]
        for h in range(3 * nf):
            corners[int(F[h // 3, h % 3])].append(h)
        bnd = np.zeros(nv, bool)
        for h in range(3 * nf):
            if twin[h] < 0:
                bnd[F[h // 3, h % 3]] = True
                bnd[F[h // 3, (h % 3 + 1) % 3]] = True
        scale = np.where(bnd, math.pi, 2.0 * math.pi) / theta
        phi = np.zeros(3 * nf)
        for v in range(nv):
            cs = corners[v]
            start = min(cs)
            if bnd[v]:   # the fan starts at the corner whose outgoing edge is a boundary edge
                for h in cs:
                    if twin[h] < 0:
                        start = h
                        break
            h, acc, seen = start, 0.0, 0
            while seen < len(cs):
                phi[h] = scale[v] * acc
                acc += ang[h // 3, h % 3]
                seen += 1
                nxt = twin[3 * (h // 3) + (h % 3 + 2) % 3]   # across the corner's incoming edge
                if nxt < 0 or nxt == start:
                    break
                h = nxt
            assert seen == len(cs), "vertex fan is not a single disk or sector"
        self.theta, self.scale, self.phi, self.bnd = theta, scale, phi.reshape(nf, 3), bnd
        # connection Laplacian: for the half-edge (f, k) from i = F[f,k] to j = F[f,k+1],
        # phi_ij = phi(f, k) and phi_ji = phi(f, k+1) + s_j * angle(f, k+1) (the edge j -> i
        # turned counter-clockwise from j's outgoing edge in the same face)
        rows, cols, vals = [], [], []
        for k in range(3):
            k1, k2 = (k + 1) % 3, (k + 2) % 3
            i, j = F[:, k], F[:, k1]
            p_ij = self.phi[:, k]
            p_ji = self.phi[:, k1] + scale[j] * ang[:, k1]
            w = 0.5 * cot[:, k2]                      # the corner opposite edge (k, k+1)
            r_ji = np.exp(1j * (p_ij + math.pi - p_ji))   # j's frame -> i's frame
            rows += [i, j, i, j]
            cols += [j, i, i, j]
            vals += [-w * r_ji, -w * np.conj(r_ji), w.astype(complex), w.astype(complex)]
        self.Lc = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(nv, nv))
        lens = np.concatenate([l01, l02, l12])
        self.h = float(np.mean(lens))
        self.t = t_factor * self.h ** 2
        self._heat = spla.splu((self.M + self.t * self.L).tocsc())
        self._vheat = spla.splu((self.M + self.t * self.Lc).tocsc())
        # Poisson with the constant gauge fixed by a Lagrange multiplier (closed meshes have
        # the constants as kernel; the right-hand side sums to zero)
        ones = sp.csr_matrix(np.ones((nv, 1)))
        A = sp.bmat([[self.L, ones], [ones.T, None]]).tocsc()
        self._pois = spla.splu(A)

    # ---- conversions between face-plane directions and vertex frames
    def to_vertex_angle(self, f, k, beta):
        """Vertex-frame angle at corner (f, k) of the face-plane direction of layout angle beta."""
        v = self.F[f, k]
        return self.phi[f, k] + self.scale[v] * _wrap(beta - self.gam[f, k])

    def grad(self, u):
        """Per-face gradient of the piecewise-linear u, in each face's layout (nf x 2)."""
        P, F = self.P, self.F
        g = np.zeros((self.nf, 2))
        for k in range(3):
            e = P[:, (k + 2) % 3] - P[:, (k + 1) % 3]        # opposite edge, counter-clockwise
            g += u[F[:, k]][:, None] * np.stack([-e[:, 1], e[:, 0]], axis=1)
        return g / (2.0 * self.area)[:, None]

    def div(self, Xf):
        """Integrated divergence at the vertices of a per-face field (layout coordinates)."""
        P, F = self.P, self.F
        out = np.zeros(self.nv)
        for k in range(3):
            k1, k2 = (k + 1) % 3, (k + 2) % 3
            e1 = P[:, k1] - P[:, k]
            e2 = P[:, k2] - P[:, k]
            c = 0.5 * (self.cot[:, k2] * np.sum(e1 * Xf, axis=1) + self.cot[:, k1] * np.sum(e2 * Xf, axis=1))
            out += np.bincount(F[:, k], weights=c, minlength=self.nv)
        return out

    # ---- the solver
    def solve(self, f0: int, b0):
        """Fields of one source (face f0, barycentrics b0): heat u, transported reference H
        (unit complex per vertex, vertex frames), unit field X per face, distance phi."""
        b0 = np.asarray(b0, np.float64)
        u0 = np.zeros(self.nv)
        Y0 = np.zeros(self.nv, complex)
        for k in range(3):
            v = self.F[f0, k]
            u0[v] += b0[k]
            Y0[v] += b0[k] * np.exp(1j * self.to_vertex_angle(f0, k, 0.0))
        u = self._heat.solve(u0)
        Y = self._vheat.solve(Y0)
        H = Y / np.abs(Y)
        g = self.grad(u)
        gn = np.linalg.norm(g, axis=1)
        with np.errstate(divide="ignore", invalid="ignore"):   # where u underflowed: X = 0
            X = np.where((gn > 0.0)[:, None], -g / gn[:, None], 0.0)
        rhs = np.concatenate([-self.div(X), [0.0]])
        phi = self._pois.solve(rhs)[:self.nv]
        phi -= float(np.dot(b0, phi[self.F[f0]]))
        return u, H, X, phi

    def evaluate(self, f0, b0, fields, tf, tb):
        """Distance and world tangent at the source towards targets (faces tf, bary tb)."""
        _, H, X, phi = fields
        tf = np.asarray(tf, np.int64)
        tb = np.asarray(tb, np.float64)
        d = np.sum(tb * phi[self.F[tf]], axis=1)
        G = self.grad(phi)[tf]
        beta = np.arctan2(G[:, 1], G[:, 0])
        z = np.zeros(len(tf), complex)
        for k in range(3):
            psi = self.to_vertex_angle(tf, k, beta)
            z += tb[:, k] * np.exp(1j * psi) * np.conj(H[self.F[tf, k]])
        th = np.angle(z)
        t = np.cos(th)[:, None] * self.E1[f0] + np.sin(th)[:, None] * self.E2[f0]
        return d, t

    def neighbors(self, face, bary, r_c: float, sources=None):
        """(row_start, j, dist, tangent) of every ordered pair (i, j), i != j, with the
        approximate distance below r_c (INFINITY: all pairs), rows in source order,
        columns in increasing j; `sources` restricts the rows (in that order)."""
        face = np.asarray(face, np.int64)
        bary = np.asarray(bary, np.float64)
        n = len(face)
        src = np.arange(n) if sources is None else np.asarray(sources, np.int64)
        rs, J, D, T = [0], [], [], []
        idx = np.arange(n)
        for i in src:
            fl = self.solve(int(face[i]), bary[i])
            d, t = self.evaluate(int(face[i]), bary[i], fl, face, bary)
            keep = (idx != i) & (d < r_c)
            J.append(idx[keep])
            D.append(d[keep])
            T.append(t[keep])
            rs.append(rs[-1] + int(keep.sum()))
        cat = lambda a, shape: np.concatenate(a) if a else np.zeros(shape)
        return (np.array(rs, np.int64), cat(J, (0,)).astype(np.int32), cat(D, (0,)), cat(T, (0, 3)).reshape(-1, 3))
