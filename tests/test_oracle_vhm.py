"""Pins of the approximate-solver oracle (heat-method distances, vector-heat transport).

The method is approximate, so its oracle is pinned by what the mathematics fixes about its
parts and by convergence to known geodesics: the cotan Laplacian's kernel and linear
precision, the mass, a parallel field in the kernel of the connection Laplacian on a flat
mesh (and the transported reference equal to it), first-order convergence of distances and
tangents to great circles on the unit sphere, and to the Euclidean ones on a flat periodic
patch, and agreement within a few percent with the exact polyhedral distances of the
window-propagation oracle on a noisy sphere.
"""
import math

import numpy as np
import pytest

import synth
from oracle import oracle as O
from oracle import vhm


def test_cotan_laplacian_kernel_linear_precision_and_mass():
    s = vhm.VhmMesh(synth.icosphere(3, 1.0, noise=0.02, seed=1))
    L = s.L.toarray()
    assert np.max(np.abs(L.sum(axis=1))) < 1e-12          # constants in the kernel
    assert np.max(np.abs(L - L.T)) == 0.0
    assert np.min(np.linalg.eigvalsh(L)) > -1e-10          # positive semi-definite
    assert s.M.diagonal().sum() == pytest.approx(s.area.sum(), rel=1e-13)
    # flat mesh: linear functions are harmonic at the interior vertices
    g = synth.grid_plane(9, 7, alternate=True)
    p = vhm.VhmMesh(g)
    inner = ~p.bnd
    for f in (g.verts[:, 0], g.verts[:, 1], 0.3 * g.verts[:, 0] - 1.7 * g.verts[:, 1] + 2.0):
        assert np.max(np.abs((p.L @ f)[inner])) < 1e-12
    # a non-linear function is not (the check has teeth)
    assert np.max(np.abs((p.L @ g.verts[:, 0] ** 2)[inner])) > 1e-3


def _reference_angles(s, m):
    """World angle (in the x-y plane) of each vertex's reference direction on a flat
    periodic patch: the outgoing edge of the corner whose frame angle is 0."""
    g = np.full(s.nv, np.nan)
    for f in range(s.nf):
        for k in range(3):
            v = s.F[f, k]
            if np.isnan(g[v]) and abs(s.phi[f, k]) < 1e-15:
                d = m.verts[s.F[f, (k + 1) % 3]] - m.verts[v]
                d[:2] -= np.round(d[:2])
                g[v] = math.atan2(d[1], d[0])
    assert not np.isnan(g).any()
    return g


def test_parallel_field_is_in_the_kernel_of_the_connection_laplacian():
    """On a flat periodic patch (every vertex flat) a globally constant direction is
    parallel: its vertex-frame representation is harmonic for the connection Laplacian.
    Carrying vectors with the conjugate phase (a plausible slip) breaks this."""
    m = synth.periodic_heightfield(12, 0, seed=1)
    s = vhm.VhmMesh(m)
    g = _reference_angles(s, m)
    for alpha in (0.0, 0.7, 2.9):
        Y = np.exp(1j * (alpha - g))
        assert np.max(np.abs(s.Lc @ Y)) < 1e-12
        wrong = s.Lc.copy()
        wrong.data = np.where(np.abs(wrong.data.imag) > 0, np.conj(wrong.data), wrong.data)
        assert np.max(np.abs(wrong @ Y)) > 1e-3


def test_transported_reference_is_constant_on_a_flat_patch():
    m = synth.periodic_heightfield(16, 0, seed=1)
    s = vhm.VhmMesh(m)
    g = _reference_angles(s, m)
    face, bary = synth.place_uniform(m, 5, 2)
    for f0, b0 in zip(face, bary):
        _, H, _, _ = s.solve(int(f0), b0)
        e = math.atan2(s.E1[f0][1], s.E1[f0][0])
        dev = np.angle(H * np.exp(1j * (g - e)))
        assert np.max(np.abs(dev)) < 1e-10


def _sphere_errors(level):
    m = synth.icosphere(level, 1.0)
    face, bary = synth.place_uniform(m, 200, 3)
    s = vhm.VhmMesh(m)
    src = [0, 1, 2]
    rs, j, d, t = s.neighbors(face, bary, math.inf, sources=src)
    x = synth.particles.world_positions(m, face, bary)
    de, te = [], []
    for row, i in enumerate(src):
        sl = slice(rs[row], rs[row + 1])
        x0 = x[i] / np.linalg.norm(x[i])
        xj = x[j[sl]] / np.linalg.norm(x[j[sl]], axis=1)[:, None]
        ex = np.arccos(np.clip(xj @ x0, -1.0, 1.0))
        tex = xj - (xj @ x0)[:, None] * x0           # great-circle direction at the source
        n0 = np.cross(s.E1[face[i]], s.E2[face[i]])
        tex -= (tex @ n0)[:, None] * n0                # in the source face's plane
        tex /= np.linalg.norm(tex, axis=1)[:, None]
        keep = ex < 2.0                                # away from the antipodal cut locus
        de.append(np.abs(d[sl] - ex)[keep])
        te.append(np.linalg.norm(t[sl] - tex, axis=1)[keep])
    return s.h, np.concatenate(de), np.concatenate(te)


def test_converges_to_great_circles_at_first_order():
    """Unit sphere, icosphere levels 2-4: distance and tangent errors against the great-circle
    ones shrink about linearly with the mesh spacing h (the paper's O(h) statement for the
    approximate method)."""
    hs, dm, tm = [], [], []
    for level in (2, 3, 4):
        h, de, te = _sphere_errors(level)
        hs.append(h)
        dm.append(de.mean())
        tm.append(te.mean())
    sd = np.polyfit(np.log(hs), np.log(dm), 1)[0]
    st = np.polyfit(np.log(hs), np.log(tm), 1)[0]
    assert 0.7 < sd < 1.6, (dm, sd)
    assert 0.7 < st < 1.6, (tm, st)
    assert dm[-1] < 0.05 and tm[-1] < 0.03


def test_flat_periodic_patch_is_close_to_euclidean():
    errs = []
    for n in (16, 32):
        m = synth.periodic_heightfield(n, 0, seed=1)
        face, bary = synth.place_uniform(m, 60, 4)
        s = vhm.VhmMesh(m)
        rs, j, d, t = s.neighbors(face, bary, math.inf, sources=[0, 1])
        x = synth.particles.world_positions(m, face, bary)
        e = []
        for row, i in enumerate([0, 1]):
            sl = slice(rs[row], rs[row + 1])
            dx = x[j[sl]] - x[i]
            dx[:, :2] -= np.round(dx[:, :2])
            r = np.linalg.norm(dx, axis=1)
            near = r < 0.35                            # off the minimum-image cut locus
            e.append(np.abs(d[sl] - r)[near])
            cos = np.sum(t[sl][near] * dx[near], axis=1) / r[near]
            assert np.median(cos) > 0.99
        errs.append(np.concatenate(e).mean())
    assert errs[1] < 0.75 * errs[0] and errs[1] < 0.02


def test_within_a_few_percent_of_exact_polyhedral_distances():
    m = synth.icosphere(4, 1.0, noise=0.02, seed=6)
    face, bary = synth.place_uniform(m, 150, 8)
    s = vhm.VhmMesh(m)
    src = [0, 5, 9]
    rs, j, d, t = s.neighbors(face, bary, 1.2, sources=src)
    rr, jr, dr, tr = O.OracleMesh(m).neighbors(face, bary, 1.2, sources=src)
    approx = {(src[r], int(j[q])): d[q] for r in range(len(src)) for q in range(rs[r], rs[r + 1])}
    rel = []
    for r in range(len(src)):
        for q in range(rr[r], rr[r + 1]):
            k = (src[r], int(jr[q]))
            if k in approx and dr[q] > 0.2:
                rel.append(abs(approx[k] - dr[q]) / dr[q])
    rel = np.array(rel)
    assert len(rel) > 50 and rel.mean() < 0.04 and np.percentile(rel, 95) < 0.1
