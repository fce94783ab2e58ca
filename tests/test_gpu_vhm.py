"""The approximate solver on the GPU (heat-method distances, vector-heat tangents) against
its FP64 oracle, element by element, through the C ABI (needs a GB300).

Both sides solve the same discrete equations (the oracle with direct sparse solves, the
GPU with Jacobi sweeps and conjugate gradients), so distances agree to 1e-9 of the larger
of the distance and the mesh spacing and tangents to 1e-7.  Cases: a noisy sphere, a
torus, a flat periodic patch, an open sheet with a hole (boundary vertices), enough
particles for several batches of sources, a finite cutoff, device output buffers, the
capacity protocol and argument errors.
"""
import math

import numpy as np
import pytest

import synth
from oracle import vhm as V

css = pytest.importorskip("paper_2404_19751_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = css.create(0)
    yield c
    c.close()


CASES = {
    "noisy_ico3_n80": lambda: (lambda m: (m,) + synth.place_uniform(m, 80, 3))(synth.icosphere(3, 1.0, noise=0.02, seed=4)),
    "torus_n60": lambda: (lambda m: (m,) + synth.place_uniform(m, 60, 5))(synth.torus(2.0, 0.7, 40, 18)),
    "flat_periodic_n50": lambda: (lambda m: (m,) + synth.place_uniform(m, 50, 6))(synth.periodic_heightfield(20, 0, seed=1)),
    "rough_periodic_n50": lambda: (lambda m: (m,) + synth.place_uniform(m, 50, 7))(synth.periodic_heightfield(24, 8, seed=2)),
    "holed_plane_n60": lambda: (lambda m: (m,) + synth.place_uniform(m, 60, 8))(synth.holed_plane(21, (0.4, 0.6, 0.4, 0.6))),
}


def _compare(g, r, h, band=0.0, r_c=math.inf):
    G = {(i, int(g[1][q])): (g[2][q], g[3][q]) for i in range(len(g[0]) - 1) for q in range(g[0][i], g[0][i + 1])}
    R = {(i, int(r[1][q])): (r[2][q], r[3][q]) for i in range(len(r[0]) - 1) for q in range(r[0][i], r[0][i + 1])}
    for k in set(G) ^ set(R):
        d = G[k][0] if k in G else R[k][0]
        assert abs(d - r_c) <= band, (k, d)
    md = mt = 0.0
    for k in set(G) & set(R):
        md = max(md, abs(G[k][0] - R[k][0]) / max(abs(R[k][0]), h))
        mt = max(mt, float(np.linalg.norm(G[k][1] - R[k][1])))
    assert md <= 1e-9, md
    assert mt <= 1e-7, mt
    return len(set(G) & set(R))


@pytest.mark.parametrize("name", list(CASES))
def test_vhm_matches_oracle_all_pairs(ctx, name):
    m, face, bary = CASES[name]()
    mesh = css.mesh_upload(ctx, m.verts, m.faces, m.period)
    parts = css.particles_set(ctx, mesh, face, bary)
    g = css.vhm_neighbors(parts, math.inf, 1.0)
    om = V.VhmMesh(m, t_factor=1.0)
    r = om.neighbors(face, bary, math.inf)
    n = _compare(g, r, om.h)
    assert n == len(face) * (len(face) - 1)
    c = ctx.last_counters()
    assert c["sources"] == len(face) and c["pairs"] == n
    parts.free()
    mesh.free()


def test_vhm_batches_cutoff_and_time_factor(ctx):
    """300 sources (two batches of 256 columns), a finite cutoff and t = 2 h^2."""
    m = synth.icosphere(3, 1.0, noise=0.01, seed=9)
    face, bary = synth.place_uniform(m, 300, 10)
    mesh = css.mesh_upload(ctx, m.verts, m.faces)
    parts = css.particles_set(ctx, mesh, face, bary)
    g = css.vhm_neighbors(parts, 0.8, 2.0)
    assert ctx.last_counters()["retries"] == 256 and ctx.last_counters()["deferred"] == 2   # columns, batches
    om = V.VhmMesh(m, t_factor=2.0)
    r = om.neighbors(face, bary, 0.8)
    assert _compare(g, r, om.h, band=1e-9, r_c=0.8) > 1000
    parts.free()
    mesh.free()


def test_vhm_device_outputs_capacity_and_errors(ctx):
    torch = pytest.importorskip("torch")
    import ctypes as C
    m = synth.torus(2.0, 0.6, 24, 12)
    face, bary = synth.place_uniform(m, 40, 11)
    mesh = css.mesh_upload(ctx, m.verts, m.faces)
    parts = css.particles_set(ctx, mesh, face, bary)
    ref = css.vhm_neighbors(parts, math.inf, 1.0)
    L = css.load()
    need = C.c_int64(0)
    assert L.css_vhm_neighbors(parts.h, math.inf, 1.0, 10, C.byref(need), None, None, None, None) == -5
    assert need.value == 40 * 39
    k = need.value
    rs = torch.zeros(41, dtype=torch.int64, device="cuda")
    j = torch.zeros(k, dtype=torch.int32, device="cuda")
    d = torch.zeros(k, dtype=torch.float64, device="cuda")
    t = torch.zeros((k, 3), dtype=torch.float64, device="cuda")
    assert L.css_vhm_neighbors(parts.h, math.inf, 1.0, k, C.byref(need), rs.data_ptr(), j.data_ptr(), d.data_ptr(),
                               t.data_ptr()) == 0
    torch.cuda.synchronize()
    assert np.array_equal(rs.cpu().numpy(), ref[0]) and np.array_equal(j.cpu().numpy(), ref[1])
    assert np.array_equal(d.cpu().numpy(), ref[2]) and np.array_equal(t.cpu().numpy(), ref[3])
    for bad in ((math.inf, 0.0), (math.inf, -1.0), (math.inf, math.nan), (math.nan, 1.0), (0.0, 1.0)):
        assert L.css_vhm_neighbors(parts.h, bad[0], bad[1], k, C.byref(need), None, None, None, None) == -1
    parts.free()
    mesh.free()


def test_vhm_is_close_to_exact_distances(ctx):
    """The approximate distances lie within a few percent of the exact window-propagation
    distances of the library itself (the paper's trade-off, Sec. 2.2)."""
    m = synth.icosphere(4, 1.0, noise=0.01, seed=12)
    face, bary = synth.place_uniform(m, 120, 13)
    mesh = css.mesh_upload(ctx, m.verts, m.faces)
    parts = css.particles_set(ctx, mesh, face, bary)
    a = css.vhm_neighbors(parts, math.inf, 1.0)
    e = css.geodesic_neighbors(parts, math.inf, css.FP64)
    assert np.array_equal(a[0], e[0]) and np.array_equal(a[1], e[1])
    far = e[2] > 0.3
    rel = np.abs(a[2] - e[2])[far] / e[2][far]
    assert rel.mean() < 0.03 and np.percentile(rel, 99) < 0.1
    cos = np.sum(a[3] * e[3], axis=1)[far & (e[2] < 2.5)]
    assert np.median(cos) > 0.99
    parts.free()
    mesh.free()
