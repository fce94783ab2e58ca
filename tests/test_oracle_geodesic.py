"""Pins of the CPU oracle's geodesic distances and tangents (no GPU).

Each test checks the oracle against something fixed independently of its code:
closed forms (flat, developable tube, cube unfoldings), the definitional
brute-force solver on tiny meshes, metric invariants, the smooth-sphere limit
and published Philox vectors.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import brute
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_normals_moments():
    z = np.array([O.normal_pair(7, i, 3) for i in range(20000)]).ravel()
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1.0) < 0.03
    assert O.normal_pair(7, 1, 3) != O.normal_pair(7, 1, 4)


def _ks_stat(x, cdf):
    """Kolmogorov-Smirnov statistic of the sample x against the distribution function cdf."""
    x = np.sort(np.asarray(x))
    n = len(x)
    F = cdf(x)
    return max(np.max(np.arange(1, n + 1) / n - F), np.max(F - np.arange(n) / n))


def test_normals_are_independent_standard_pairs():
    """The two normals of one Philox draw are an independent standard pair (Box-Muller):
    each is N(0, 1), they are uncorrelated, z0^2 + z1^2 is exponential with mean 2 and the
    angle atan2(z1, z0) is uniform.  A mix-up of cos and sin (z1 equal to z0, or to -z0), a
    wrong radius or a missing 2 pi each fail one of these at the 0.1 % KS level."""
    n = 20000
    z = np.array([O.normal_pair(11, i, 5) for i in range(n)])
    z0, z1 = z[:, 0], z[:, 1]
    crit = 1.95 / math.sqrt(n)   # KS critical value at the 0.1 % level
    phi = np.vectorize(lambda t: 0.5 * (1.0 + math.erf(t / math.sqrt(2.0))))
    assert _ks_stat(z0, phi) < crit
    assert _ks_stat(z1, phi) < crit
    assert abs(np.corrcoef(z0, z1)[0, 1]) < 4.0 / math.sqrt(n)
    assert _ks_stat(z0 ** 2 + z1 ** 2, lambda r: 1.0 - np.exp(-0.5 * r)) < crit
    assert _ks_stat(np.arctan2(z1, z0), lambda a: (a + math.pi) / (2.0 * math.pi)) < crit
    # consecutive steps of one particle are independent draws too
    w = np.array([O.normal_pair(11, 3, s)[0] for s in range(n)])
    assert abs(np.corrcoef(w[:-1], w[1:])[0, 1]) < 4.0 / math.sqrt(n)


def test_flat_plane_is_euclidean():
    """Open flat convex mesh: geodesic = straight segment, tangent = unit chord (Sec. 2.1)."""
    cfg = synth.make_config("flat64")
    m, face, bary = cfg["mesh"], cfg["face"], cfg["bary"]
    om = O.OracleMesh(m)
    x = synth.particles.world_positions(m, face, bary)
    rs, j, d, t = om.neighbors(face, bary, math.inf)
    assert rs[-1] == 64 * 63
    for i in range(64):
        jj = j[rs[i]:rs[i + 1]]
        dx = x[jj] - x[i]
        e = np.linalg.norm(dx, axis=1)
        np.testing.assert_allclose(d[rs[i]:rs[i + 1]], e, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(t[rs[i]:rs[i + 1]], dx / e[:, None], atol=1e-12)


def _tube_coords(m, x):
    n = m.meta["n_around"]
    rho = m.meta["radius"]
    side = 2 * rho * math.sin(math.pi / n)
    phi = np.mod(np.arctan2(x[:, 1], x[:, 0]), 2 * np.pi)
    i = np.minimum(np.floor(phi / (2 * np.pi / n)).astype(int), n - 1)
    a0 = 2 * np.pi * i / n
    a1 = 2 * np.pi * (i + 1) / n
    v0 = np.stack([rho * np.cos(a0), rho * np.sin(a0)], 1)
    v1 = np.stack([rho * np.cos(a1), rho * np.sin(a1)], 1)
    t = np.linalg.norm(x[:, :2] - v0, axis=1) / side
    e = (v1 - v0) / side
    return (i + t) * side, x[:, 2], n * side, np.concatenate([e, np.zeros((len(x), 1))], 1)


def test_tube_is_unrolled_with_wraps():
    """Developable open prism tube: d = min_k |(du + k P, dz)| in the unrolled strip."""
    m = synth.cylinder_tube(9, 5, 1.0, 2.5)
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 40, 11)
    x = synth.particles.world_positions(m, face, bary)
    u, z, P, eside = _tube_coords(m, x)
    rs, j, d, t = om.neighbors(face, bary, math.inf)
    for i in range(len(face)):
        jj = j[rs[i]:rs[i + 1]]
        du = u[jj] - u[i]
        cands = np.stack([np.hypot(du + k * P, z[jj] - z[i]) for k in (-1, 0, 1)], 1)
        kbest = np.argmin(cands, 1)
        np.testing.assert_allclose(d[rs[i]:rs[i + 1]], cands.min(1), rtol=1e-11)
        srt = np.sort(cands, 1)
        clear = srt[:, 1] - srt[:, 0] > 1e-6
        dub = du + np.array([-1, 0, 1])[kbest] * P
        tt = (dub[:, None] * eside[i] + (z[jj] - z[i])[:, None] * np.array([0, 0, 1.0])) / cands.min(1)[:, None]
        np.testing.assert_allclose(t[rs[i]:rs[i + 1]][clear], tt[clear], atol=1e-9)


def _locate(m, pt):
    P = m.verts[m.faces]
    for f in range(m.nf):
        A, B, C = P[f]
        n = np.cross(B - A, C - A)
        n /= np.linalg.norm(n)
        if abs(np.dot(pt - A, n)) > 1e-12:
            continue
        M = np.stack([B - A, C - A], 1)
        l = np.linalg.lstsq(M, pt - A, rcond=None)[0]
        b = np.array([1 - l.sum(), l[0], l[1]])
        if b.min() > -1e-12:
            return f, np.clip(b, 0, 1) / np.clip(b, 0, 1).sum()
    raise ValueError(pt)


def test_cube_unfoldings():
    """Unit cube: lengths of explicit unfoldings; corners (angle sum 3 pi/2) are never crossed."""
    m = synth.cube(2)
    om = O.OracleMesh(m)
    th, ps, bd = om.vertex_info()
    corners = np.isclose(th, 1.5 * np.pi)
    assert corners.sum() == 8 and not ps[corners].any() and ps[~corners].all()
    src = np.array([0.5, 0.4, 1.0])
    tg = {  # point: closed-form unfolded length
        (0.5, 0.4, 0.0): 0.4 + 1.0 + 0.4,                 # over the y=0 side
        (1.0, 0.5, 0.4): math.hypot(1.1, 0.1),            # top + x=1 side
        (0.4, 0.0, 0.5): math.hypot(0.1, 0.9),            # top + y=0 side
        (0.5, 0.5, 0.0): 2.0 - 0.1,                        # over y=0: 0.4 + 1 + 0.5
    }
    f0, b0 = _locate(m, src)
    fb = [_locate(m, np.array(p)) for p in tg]
    d, t = om.query(f0, b0, math.inf, [f for f, _ in fb], [b for _, b in fb])
    np.testing.assert_allclose(d, list(tg.values()), rtol=1e-13)
    # face centre to face centre: adjacent sides 1, opposite sides 2 (sources on vertices)
    c_top, c_side, c_bot = (0.5, 0.5, 1.0), (1.0, 0.5, 0.5), (0.5, 0.5, 0.0)
    f0, b0 = _locate(m, np.array(c_top))
    fb = [_locate(m, np.array(c)) for c in (c_side, c_bot)]
    d, _ = om.query(f0, b0, math.inf, [f for f, _ in fb], [b for _, b in fb])
    np.testing.assert_allclose(d, [1.0, 2.0], rtol=1e-13)


def test_periodic_flat_patch_is_minimum_image():
    """Periodic flat square: geodesic = minimum-image Euclidean distance below half the period."""
    m = synth.periodic_heightfield(24, 1, seed=0, A=(0.0, 0.0))
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 30, 5)
    x = synth.particles.world_positions(m, face, bary)
    rs, j, d, t = om.neighbors(face, bary, 0.45)
    n_checked = 0
    for i in range(len(face)):
        dx = x - x[i]
        dx[:, :2] -= np.round(dx[:, :2])
        e = np.linalg.norm(dx, axis=1)
        want = np.where((e < 0.45) & (np.arange(len(face)) != i))[0]
        assert list(j[rs[i]:rs[i + 1]]) == list(want)
        np.testing.assert_allclose(d[rs[i]:rs[i + 1]], e[want], rtol=1e-12)
        np.testing.assert_allclose(t[rs[i]:rs[i + 1]], dx[want] / e[want, None], atol=1e-11)
        n_checked += len(want)
    assert n_checked > 100


TINY = [
    ("tetra", lambda: synth.tetrahedron()),
    ("octa", lambda: synth.octahedron()),
    ("cube1", lambda: synth.cube(1)),
    ("cube2", lambda: synth.cube(2)),
    ("torus8x5", lambda: synth.torus(3, 1, 8, 5)),
    ("noisy_ico1", lambda: synth.icosphere(1, 1.0, noise=0.15, seed=3)),
    ("plane4", lambda: synth.grid_plane(4, 4, alternate=True)),
    ("tube6x3", lambda: synth.cylinder_tube(6, 3, 1.0, 2.0)),
]


@pytest.mark.parametrize("name,make", TINY, ids=[t[0] for t in TINY])
def test_window_propagation_matches_brute_force(name, make):
    """O-mmp == definitional unfold-and-Dijkstra solver on tiny meshes (Sec. 2.2)."""
    m = make()
    om = O.OracleMesh(m)
    n = 6
    face, bary = synth.place_uniform(m, n, 0)
    dmax = 1.5 * synth.bbox_diagonal(m)
    for i in range(n):
        db, tb = brute.geodesics(m, face[i], bary[i], list(zip(face, bary)), dmax)
        do, to = om.query(face[i], bary[i], math.inf, face, bary)
        mask = np.arange(n) != i
        np.testing.assert_allclose(do[mask], db[mask], rtol=1e-12)
        np.testing.assert_allclose(to[mask], tb[mask], atol=1e-9)


def test_noisy_sphere_invariants():
    """Symmetry, triangle inequality, Euclidean lower bound (Sec. 3.1), unit tangents."""
    m = synth.icosphere(2, 1.0, noise=0.04, seed=9)
    om = O.OracleMesh(m)
    th, ps, _ = om.vertex_info()
    assert ps.sum() > 10                      # saddle vertices exist
    face, bary = synth.place_uniform(m, 40, 4)
    x = synth.particles.world_positions(m, face, bary)
    rs, j, d, t = om.neighbors(face, bary, math.inf)
    n = len(face)
    D = np.full((n, n), 0.0)
    for i in range(n):
        D[i, j[rs[i]:rs[i + 1]]] = d[rs[i]:rs[i + 1]]
    np.testing.assert_allclose(D, D.T, rtol=1e-12, atol=1e-14)
    E = np.linalg.norm(x[:, None] - x[None], axis=2)
    assert (D >= E - 1e-12).all()
    tri = D[:, None, :] <= D[:, :, None] + D[None, :, :] + 1e-12
    assert tri.all()
    np.testing.assert_allclose(np.linalg.norm(t, axis=1), 1.0, atol=1e-12)


def test_cutoff_is_a_filter():
    """A cutoff only removes pairs (Sec. 3.1 submeshing): same distances below r_c."""
    m = synth.icosphere(3, 1.0, noise=0.01, seed=2)
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 60, 8)
    rs0, j0, d0, t0 = om.neighbors(face, bary, math.inf)
    for rc in (0.3, 0.7):
        rs, j, d, t = om.neighbors(face, bary, rc)
        for i in range(len(face)):
            keep = d0[rs0[i]:rs0[i + 1]] < rc
            assert list(j[rs[i]:rs[i + 1]]) == list(j0[rs0[i]:rs0[i + 1]][keep])
            np.testing.assert_allclose(d[rs[i]:rs[i + 1]], d0[rs0[i]:rs0[i + 1]][keep], rtol=1e-13)
            np.testing.assert_allclose(t[rs[i]:rs[i + 1]], t0[rs0[i]:rs0[i + 1]][keep], atol=1e-12)


def test_sphere_converges_to_great_circle():
    """Icosphere distances approach great-circle arcs as the mesh refines (Sec. 2.2, O(h^2))."""
    errs = []
    for level in (2, 3, 4):
        m = synth.icosphere(level, 1.0)
        om = O.OracleMesh(m)
        face, bary = synth.place_uniform(m, 12, 1)
        x = synth.particles.world_positions(m, face, bary)
        u = x / np.linalg.norm(x, axis=1, keepdims=True)
        rs, j, d, t = om.neighbors(face, bary, 1.5)
        e = 0.0
        for i in range(len(face)):
            jj = j[rs[i]:rs[i + 1]]
            arc = np.arccos(np.clip(u[jj] @ u[i], -1, 1))
            e = max(e, np.max(np.abs(d[rs[i]:rs[i + 1]] - arc)))
        errs.append(e)
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 2.5           # close to 4 for a second-order error


def test_mesh_validation():
    m = synth.tetrahedron()
    bad = m.faces.copy()
    bad[0] = bad[0][[0, 2, 1]]               # one face flipped
    with pytest.raises(ValueError):
        O.OracleMesh(synth.meshes.Mesh(m.verts, bad))
    three = np.concatenate([m.faces, [[0, 1, 3]]])  # edge (0,1) used three times
    with pytest.raises(ValueError):
        O.OracleMesh(synth.meshes.Mesh(m.verts, three))


def test_walk_check_rejects_a_wrong_tangent():
    """The cut-locus acceptance rule used by the GPU parity tests (a differing tangent must
    start a geodesic of the reported length to the target) rejects a perturbed tangent."""
    from tests._common import geodesic_walker
    m = synth.icosphere(3, 1.0)
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 30, 4)
    rs, j, d, t = om.neighbors(face, bary, 0.5)
    walk = geodesic_walker(om, face, bary)
    fr = om.face_frame(face[0])
    n = np.cross(fr[1], fr[2])
    for q in range(rs[0], rs[1]):
        assert walk(0, int(j[q]), d[q], t[q]) < 1e-12
        bad = t[q] * math.cos(1e-3) + np.cross(n, t[q]) * math.sin(1e-3)
        assert walk(0, int(j[q]), d[q], bad) > 1e-5 * d[q]


def test_descent_check_accepts_shortest_directions_only():
    """First-variation check used for cut-locus tangents: 0 deficit along a true initial
    tangent (also for paths bending at saddle vertices), 1 - cos(angle) off it."""
    from tests._common import descent_checker
    m = synth.icosphere(2, 1.0, noise=0.05, seed=9)
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 30, 4)
    rs, j, d, t = om.neighbors(face, bary, 1.0)
    chk = descent_checker(om, face, bary, 1.0)
    for i in (0, 1, 2):
        fr = om.face_frame(face[i])
        n = np.cross(fr[1], fr[2])
        for q in range(rs[i], rs[i + 1]):
            assert abs(chk(i, int(j[q]), d[q], t[q])) < 1e-8
            bad = t[q] * math.cos(2e-3) + np.cross(n, t[q]) * math.sin(2e-3)
            assert chk(i, int(j[q]), d[q], bad) > 1e-6


# ------------------------------------------------------------------ path polylines
def _locate_xy(m, x, y):
    """(face, bary) of the point (x, y, 0) of a flat mesh."""
    P = synth.meshes.unwrapped_face_vertices(m)
    for f in range(m.nf):
        A = np.array([[P[f][1][0] - P[f][0][0], P[f][2][0] - P[f][0][0]],
                      [P[f][1][1] - P[f][0][1], P[f][2][1] - P[f][0][1]]])
        l1, l2 = np.linalg.solve(A, [x - P[f][0][0], y - P[f][0][1]])
        b = np.array([1 - l1 - l2, l1, l2])
        if b.min() > 1e-9:
            return np.array([f], np.int32), b[None, :]
    raise ValueError((x, y))


def test_trace_on_a_plane_is_the_straight_segment():
    """On a flat grid the traced path is the straight segment: every recorded point lies on
    it, in order, and the crossings of the axis-parallel grid lines sit where the segment
    meets them."""
    m = synth.grid_plane(11, 11, 0, 1, 0, 1)
    om = O.OracleMesh(m)
    face, bary = _locate_xy(m, 0.213, 0.247)
    x0 = om.world(face, bary)[0]
    d = np.array([0.51, 0.37, 0.0])
    pts, n, f1, b1 = om.trace(int(face[0]), bary[0], d)
    assert n == len(pts) >= 3
    np.testing.assert_allclose(pts[0], x0, atol=1e-14)
    np.testing.assert_allclose(pts[-1], x0 + d, atol=1e-12)
    u = d / np.linalg.norm(d)
    s = (pts - x0) @ u
    assert np.all(np.diff(s) >= -1e-14)                             # in order along the segment
    np.testing.assert_allclose(np.linalg.norm((pts - x0) - np.outer(s, u), axis=1), 0, atol=1e-12)
    assert np.linalg.norm(np.diff(pts, axis=0), axis=1).sum() == pytest.approx(np.linalg.norm(d), rel=1e-12)
    # every crossing of a vertical grid line x = k/10 inside the segment is a recorded point
    for k in range(11):
        xk = k / 10
        if min(x0[0], x0[0] + d[0]) < xk < max(x0[0], x0[0] + d[0]):
            t = (xk - x0[0]) / d[0]
            assert np.min(np.linalg.norm(pts - (x0 + t * d), axis=1)) < 1e-12


def test_trace_on_a_tube_is_the_unrolled_line():
    """Around an open tube the path is a helix, straight in the unrolled strip: its points
    have arc length (unrolled) proportional to height, and the total unrolled length is the
    requested one."""
    R, H = 1.0, 2.0
    m = synth.cylinder_tube(24, 8, R, H)
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 1, 9)
    x0 = om.world(face, bary)[0]
    # a tangent direction at x0: mix of the axial and the circumferential direction
    fr = om.face_frame(int(face[0]))
    n3 = np.cross(fr[1], fr[2])
    n3 /= np.linalg.norm(n3)
    ax = np.array([0.0, 0.0, 1.0]) - np.dot([0.0, 0.0, 1.0], n3) * n3
    ax /= np.linalg.norm(ax)
    circ = np.cross(n3, ax)
    d = 1.5 * (0.6 * circ + 0.8 * ax) / np.linalg.norm(0.6 * circ + 0.8 * ax)
    if x0[2] + d[2] > H - 0.05 or x0[2] + d[2] < 0.05:
        d[2] = -d[2]
        d = 1.5 * (0.6 * circ - 0.8 * ax) / np.linalg.norm(0.6 * circ - 0.8 * ax)
    pts, n, f1, b1 = om.trace(int(face[0]), bary[0], d)
    seg = np.linalg.norm(np.diff(pts, axis=0), axis=1)
    # consecutive points share a flat face, so the polyline is the path itself
    assert seg.sum() == pytest.approx(1.5, rel=1e-12)
    dz = np.diff(pts[:, 2])
    # straight in the unrolled strip: equal height gain per unit of unrolled length
    assert np.allclose(dz / np.maximum(seg, 1e-300), dz[0] / seg[0], atol=1e-9) or np.all(np.abs(dz) < 1e-15)


def _point_to_polyline(p, Q):
    """distance from point p to the polyline through the points Q"""
    best = math.inf
    for a, b in zip(Q[:-1], Q[1:]):
        ab = b - a
        t = np.clip(np.dot(p - a, ab) / np.dot(ab, ab), 0.0, 1.0)
        best = min(best, float(np.linalg.norm(p - (a + t * ab))))
    return best


def _taut_string(S, E, lo, hi):
    """Shortest path from S to E in the plane around the open square (lo, hi)^2: the
    shortest path in the visibility graph of S, E and the square's corners (the textbook
    construction for Euclidean shortest paths among polygonal obstacles).  A segment is
    visible if no part of positive length lies inside the open square (Liang-Barsky clip)."""
    corners = [np.array([lo, lo, 0.0]), np.array([lo, hi, 0.0]), np.array([hi, hi, 0.0]), np.array([hi, lo, 0.0])]
    nodes = [S] + corners + [E]

    def visible(P, Q):
        t0, t1 = 0.0, 1.0
        for a in range(2):
            d = Q[a] - P[a]
            if abs(d) < 1e-300:
                if not (lo < P[a] < hi):
                    return True
                continue
            u0, u1 = sorted(((lo - P[a]) / d, (hi - P[a]) / d))
            t0, t1 = max(t0, u0), min(t1, u1)
        return t1 - t0 <= 1e-12

    n = len(nodes)
    dist = [math.inf] * n
    prev = [-1] * n
    dist[0] = 0.0
    done = [False] * n
    for _ in range(n):
        u = min((k for k in range(n) if not done[k]), key=lambda k: dist[k])
        done[u] = True
        for v in range(n):
            if not done[v] and visible(nodes[u], nodes[v]):
                w = dist[u] + float(np.linalg.norm(nodes[v] - nodes[u]))
                if w < dist[v]:
                    dist[v], prev[v] = w, u
    chain, k = [], n - 1
    while k >= 0:
        chain.append(nodes[k])
        k = prev[k]
    return np.array(chain[::-1]), dist[-1]


def test_paths_around_a_square_hole_are_the_taut_strings():
    """On a flat sheet with a square hole the shortest path is the taut string around the
    hole (Sec. 2.2: it bends at boundary vertices only).  Checks the distance against the
    visibility-graph shortest path, every polyline point on that string, its wrapped corners
    among the points, the polyline length, and that each leg lands on its node."""
    m = synth.holed_plane(21, (0.4, 0.6, 0.4, 0.6))
    om = O.OracleMesh(m)
    ends = [((0.43, 0.31), (0.47, 0.78)),     # two bends, left of the hole
            ((0.31, 0.52), (0.57, 0.71)),     # one bend at the upper left corner
            ((0.71, 0.47), (0.37, 0.64)),     # one bend at the upper right corner
            ((0.72, 0.33), (0.27, 0.69)),     # two bends, along the top side or the bottom side
            ((0.62, 0.33), (0.66, 0.62))]     # in sight of each other: straight
    bends = []
    for s, e in ends:
        fs, bs = _locate_xy(m, *s)
        fe, be = _locate_xy(m, *e)
        face, bary = np.concatenate([fs, fe]), np.concatenate([bs, be])
        S, E = np.array(s + (0.0,)), np.array(e + (0.0,))
        Q, L = _taut_string(S, E, 0.4, 0.6)
        paths, legs, dist, gap = om.geodesic_paths(face, bary, math.inf, [0], [1])
        assert dist[0] == pytest.approx(L, rel=1e-13, abs=1e-15)
        P = paths[0]
        np.testing.assert_allclose(P[0], S, atol=1e-14)
        np.testing.assert_allclose(P[-1], E, atol=1e-14)
        assert max(_point_to_polyline(p, Q) for p in P) < 1e-13
        for c in Q[1:-1]:
            assert np.min(np.linalg.norm(P - c, axis=1)) < 1e-13
        assert np.sum(np.linalg.norm(np.diff(P, axis=0), axis=1)) == pytest.approx(L, rel=1e-13)
        assert legs[0] >= len(Q) - 1 and gap[0] < 1e-13
        bends.append(len(Q) - 2)
    assert sorted(set(bends)) == [0, 1, 2]


def test_straight_paths_are_the_straightest_walk():
    """A path with one leg (no bend) is the straightest walk from the source along the
    pair's tangent for the pair's distance (Sec. 3.2): the same points as the face walk
    that moves particles, which is a separate routine."""
    cfg = synth.make_config("ico5_n1024")
    m, face, bary, r_c = cfg["mesh"], cfg["face"], cfg["bary"], cfg["r_c"]
    om = O.OracleMesh(m)
    src = np.array([3, 400, 777])
    rs, j, d, t = om.neighbors(face, bary, r_c, sources=src)[:4]
    S = np.repeat(src, np.diff(rs)).astype(np.int32)
    paths, legs, dist, gap = om.geodesic_paths(face, bary, r_c, S, j)
    assert np.all(legs == 1) and len(S) > 10
    np.testing.assert_allclose(dist, d, rtol=0, atol=0)
    for p in range(len(S)):
        pts, n, _, _ = om.trace(int(face[S[p]]), bary[S[p]], d[p] * t[p])
        assert len(pts) == len(paths[p])
        np.testing.assert_allclose(paths[p], pts, atol=1e-12)


def test_bent_paths_on_a_noisy_sphere_land_on_their_nodes():
    """On a noisy sphere many shortest paths bend at saddle vertices.  Every leg, walked
    straight from its node along the recorded direction for the recorded length, ends on
    the next node; the polyline (consecutive points share a face) is as long as the
    distance, starts at the source and ends at the neighbour."""
    m = synth.icosphere(4, 1.0, noise=0.04, seed=7)
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 200, 8)
    r_c = 0.5
    src = np.arange(0, 200, 20)
    rs, j, d = om.neighbors(face, bary, r_c, sources=src)[:3]
    S = np.repeat(src, np.diff(rs)).astype(np.int32)
    paths, legs, dist, gap = om.geodesic_paths(face, bary, r_c, S, j, cap=4096)
    np.testing.assert_array_equal(dist, d)
    assert np.sum(legs >= 2) > 10            # the sample holds bent paths
    assert np.max(gap) < 1e-12
    x = om.world(face, bary)
    for p in range(len(S)):
        P = paths[p]
        np.testing.assert_allclose(P[0], x[S[p]], atol=1e-13)
        np.testing.assert_allclose(P[-1], x[j[p]], atol=1e-13)
        assert np.sum(np.linalg.norm(np.diff(P, axis=0), axis=1)) == pytest.approx(d[p], rel=1e-12)


def test_holed_sheet_distances_are_the_visibility_graph_distances():
    """All pairs of 24 random points of a flat sheet with a square hole: the window
    propagation's distances (boundary vertices act as pseudo-sources) equal the
    visibility-graph shortest paths around the hole to 1e-12, and every pair's polyline
    lands on its nodes."""
    m = synth.holed_plane(21, (0.4, 0.6, 0.4, 0.6))
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 24, 17)
    x = om.world(face, bary)
    rs, j, d = om.neighbors(face, bary, math.inf)[:3]
    src = np.repeat(np.arange(len(face)), np.diff(rs))
    assert len(j) == 24 * 23
    for k in range(len(j)):
        _, L = _taut_string(x[src[k]], x[j[k]], 0.4, 0.6)
        assert d[k] == pytest.approx(L, rel=1e-12, abs=1e-15)
    paths, legs, dist, gap = om.geodesic_paths(face, bary, math.inf, src.astype(np.int32), j)
    assert np.max(gap) < 1e-13 and np.sum(legs >= 2) > 20


def _fan_point(m, r, phi):
    """(face, bary) of the point at intrinsic polar coordinates (r, phi) around the apex of
    a saddle fan (phi counted across the sectors, each sector pi/3 wide)."""
    rim = m.meta["rim"]
    k = len(rim)
    s = int(phi // (math.pi / 3)) % k
    psi = phi - s * math.pi / 3
    p = r * (math.sin(math.pi / 3 - psi) * rim[s] + math.sin(psi) * rim[(s + 1) % k]) / math.sin(math.pi / 3)
    best = None
    for f, tri in enumerate(m.verts[m.faces]):
        A = np.stack([tri[1] - tri[0], tri[2] - tri[0]], axis=1)
        l, res, *_ = np.linalg.lstsq(A, p - tri[0], rcond=None)
        b = np.array([1 - l.sum(), l[0], l[1]])
        err = np.linalg.norm(A @ l - (p - tri[0]))
        if b.min() > -1e-12 and err < 1e-12 and (best is None or b.min() > best[2].min()):
            best = (f, p, b)
    return best


def test_saddle_vertex_distances_and_bends_are_the_cone_closed_form():
    """An interior saddle vertex: a fan of 8 equilateral triangles has total angle 8 pi/3 at
    its apex, a cone whose developed angle exceeds 2 pi.  Two points at intrinsic radii r1,
    r2 and angular separation D (the smaller of the two ways round) are straight apart,
    sqrt(r1^2 + r2^2 - 2 r1 r2 cos D), when D < pi; otherwise the shortest path bends at the
    apex and is r1 + r2 long (Sec. 2.2: shortest paths bend only at saddle or boundary
    vertices).  Checks the distances of all pairs, one leg or two legs meeting at the apex,
    and the polyline length."""
    m = synth.saddle_fan(8, 4)
    om = O.OracleMesh(m)
    theta = 8 * math.pi / 3
    rng = np.random.default_rng(21)
    pts = [(rng.uniform(0.1, 0.45), rng.uniform(0.0, theta)) for _ in range(14)]
    loc = [_fan_point(m, r, ph) for r, ph in pts]
    face = np.array([l[0] for l in loc], np.int32)
    bary = np.array([l[2] for l in loc])
    rs, j, d = om.neighbors(face, bary, math.inf)[:3]
    src = np.repeat(np.arange(len(pts)), np.diff(rs))
    paths, legs, dist, gap = om.geodesic_paths(face, bary, math.inf, src.astype(np.int32), j)
    bent = 0
    for k in range(len(j)):
        (r1, p1), (r2, p2) = pts[src[k]], pts[j[k]]
        D = abs(p1 - p2) % theta
        D = min(D, theta - D)
        L = r1 + r2 if D >= math.pi else math.sqrt(r1 * r1 + r2 * r2 - 2 * r1 * r2 * math.cos(D))
        assert d[k] == pytest.approx(L, rel=1e-12)
        assert np.sum(np.linalg.norm(np.diff(paths[k], axis=0), axis=1)) == pytest.approx(L, rel=1e-12)
        if D > math.pi + 1e-6:
            bent += 1
            assert legs[k] == 2 and np.min(np.linalg.norm(paths[k], axis=1)) < 1e-13   # through the apex
        elif D < math.pi - 1e-6:
            assert legs[k] == 1
    assert bent >= 20 and np.max(gap) < 1e-13


def _grid16_point(x, y):
    """Face and barycentrics of (x, y) on grid_plane(17, 17) (spacing 1/16, quads split along
    the rising diagonal); exact for coordinates that are multiples of 1/64."""
    i, j = int(16 * x), int(16 * y)
    u, v = 16 * x - i, 16 * y - j
    q = j * 16 + i
    if v <= u:   # below the diagonal: corners (a, b, d)
        return 2 * q, (1.0 - u, u - v, v)
    return 2 * q + 1, (1.0 - v, u, v - u)   # above: corners (a, d, c)


def flat_vertex_pair():
    """A flat sheet with 30 particles; particles 0 and 1 lie on a line through the interior
    vertex (1/2, 1/2), all coordinates exact binary fractions, so the shortest path between
    them passes through the vertex exactly."""
    m = synth.grid_plane(17, 17)
    face, bary = synth.place_uniform(m, 30, 21, area_weighted=False)
    for k, (x, y) in enumerate(((29 / 64, 31 / 64), (41 / 64, 35 / 64))):
        f, b = _grid16_point(x, y)
        face[k], bary[k] = f, b
    return m, face, bary, np.array([0.5, 0.5, 0.0])


def test_path_through_a_flat_vertex_is_the_straight_segment():
    """A shortest path that meets an interior flat vertex exactly goes straight through it: the
    polyline lies on the segment between the two particles, contains the vertex and is as
    long as the Euclidean distance (the pass-straight rule at angle pi, pinned by the plane's
    closed form rather than by the walk's own arithmetic)."""
    m, face, bary, V = flat_vertex_pair()
    om = O.OracleMesh(m)
    x = synth.particles.world_positions(m, face, bary)
    P, Q = x[0], x[1]
    assert np.linalg.norm(np.cross(Q - P, V - P)) < 1e-15          # collinear by construction
    for s, d in ((0, 1), (1, 0)):
        paths, legs, dist, gap = om.geodesic_paths(face, bary, math.inf, [s], [d])
        pts = paths[0]
        a, b = x[s], x[d]
        assert dist[0] == pytest.approx(np.linalg.norm(b - a), rel=1e-13)
        u = (b - a) / np.linalg.norm(b - a)
        off = np.linalg.norm(np.cross(pts - a, u), axis=1)
        assert off.max() < 1e-12
        assert np.min(np.linalg.norm(pts - V, axis=1)) < 1e-12      # the vertex is on the polyline
        proj = (pts - a) @ u
        assert np.all(np.diff(proj) >= -1e-12)                       # monotone along the segment
        assert np.linalg.norm(pts[0] - a) < 1e-12 and np.linalg.norm(pts[-1] - b) < 1e-12
