"""CUDA path vs CPU oracle at the full workload sizes, on sampled outputs (needs a GB300).

The GPU computes every source of the workload in one launch, exactly as the benchmark
times it; the oracle then computes a seeded sample of the same rows one by one and the two
are compared element by element with the tolerances of the small-size parity tests:

  * periodic Gaussian height field, 256 x 256 grid (131072 faces), 8192 particles,
    r_c = 0.05, WCA;
  * noisy icosphere level 8, radius 10 (1310720 faces), 65536 particles, r_c = 2^(1/6) 0.2,
    WCA;
  * 64 tori of 2k-60k faces with 128-4096 particles each, r_c = 0.1, harmonic, advanced
    together by the batched form (one persistent launch per step inside a CUDA graph).
"""
import math

import numpy as np
import pytest

import synth
from oracle import oracle as O
from tests._common import (FP32_REL_DIAM, FP64_RTOL, compare_pairs, descent_checker, force_row_bounds,
                           sample_sources, select_rows)

css = pytest.importorskip("paper_2404_19751_gb300")
pytestmark = pytest.mark.gpu

N_SAMPLE = 48


@pytest.fixture(scope="module")
def ctx():
    c = css.create(0)
    yield c
    c.close()


@pytest.fixture(scope="module", params=["hfield256_n8192", "noisy_ico8_n65536"])
def workload(request, ctx):
    cfg = synth.make_config(request.param)
    m = cfg["mesh"]
    mesh = css.mesh_upload(ctx, m.verts, m.faces, m.period)
    parts = css.particles_set(ctx, mesh, cfg["face"], cfg["bary"], cfg["vel"], cfg["orient"], seed=5)
    om = O.OracleMesh(m)
    src = sample_sources(len(cfg["face"]), N_SAMPLE, 11)
    yield cfg, mesh, parts, om, src
    parts.free()
    mesh.free()


def test_full_size_rows_fp64(workload):
    cfg, mesh, parts, om, src = workload
    face, bary, r_c = cfg["face"], cfg["bary"], cfg["r_c"]
    g = css.geodesic_neighbors(parts, r_c, css.FP64)
    r = om.neighbors_gap(face, bary, r_c, sources=src)
    n, md, mt = compare_pairs(select_rows(g, src), r, r_c, FP64_RTOL, 1e-7)
    assert n > N_SAMPLE
    # every row, not only the sampled ones: symmetric, above the Euclidean distance, < r_c
    rs, j, d, _ = g
    assert np.all(d < r_c)
    pairs = {}
    for i in range(len(rs) - 1):
        for q in range(rs[i], rs[i + 1]):
            pairs[(i, int(j[q]))] = float(d[q])
    x = synth.particles.world_positions(cfg["mesh"], face, bary)
    for (i, k), dik in pairs.items():
        if (k, i) in pairs:
            assert abs(pairs[(k, i)] - dik) <= 1e-9 * dik
        else:
            assert abs(dik - r_c) <= 1e-9 * r_c
    dx = x[np.repeat(np.arange(len(rs) - 1), np.diff(rs))] - x[j]
    if cfg["mesh"].period is not None:
        per = np.array(list(cfg["mesh"].period) + [math.inf])
        dx[:, :2] -= np.round(dx[:, :2] / per[:2]) * per[:2]
    assert np.all(d >= np.linalg.norm(dx, axis=1) * (1 - 1e-9))


def test_full_size_rows_fp32(workload):
    cfg, mesh, parts, om, src = workload
    face, bary, r_c = cfg["face"], cfg["bary"], cfg["r_c"]
    tol = FP32_REL_DIAM * synth.bbox_diagonal(cfg["mesh"])
    g = css.geodesic_neighbors(parts, r_c, css.FP32)
    r = om.neighbors_gap(face, bary, r_c, sources=src)
    gs = select_rows(g, src)
    # row indices of the sample are local to the sample; the descent check wants particle ids
    walker = descent_checker(om, face, bary, r_c)
    n, md, mt = compare_pairs(gs, r, r_c, tol, 1e-5, rel=False, band=tol, tie=tol,
                              walker=lambda i, j, d, t: walker(int(src[i]), j, d, t), land_tol=1e-7)
    assert n > N_SAMPLE
    assert len(g[1]) == len(css.geodesic_neighbors(parts, r_c, css.FP64)[1])


def test_full_size_rows_in_the_tuned_shapes(workload, ctx):
    """The shapes the autotuner picks for these workloads in the benchmark (global tables,
    32768-window pools, the 128-register variant with 8 warps per CTA, and the first pass
    with shared tables at scale 4) give the same pairs as the default shape, with distances
    and tangents equal up to FP32 rounding."""
    cfg, mesh, parts, om, src = workload
    r_c = cfg["r_c"]
    before = ctx.get_launch()
    ref = css.geodesic_neighbors(parts, r_c, css.FP32)
    for shape in (dict(warps_per_cta=8, ctas_per_sm=0, tile=1, shared_scale=0, window_capacity=32768,
                       window_capacity2=16384, warps2_per_sm=2, occupancy=2),
                  dict(warps_per_cta=2, ctas_per_sm=0, tile=1, shared_scale=4, window_capacity=8192,
                       window_capacity2=16384, warps2_per_sm=2, occupancy=1)):
        ctx.set_launch(**shape)
        g = css.geodesic_neighbors(parts, r_c, css.FP32)
        assert np.array_equal(g[0], ref[0]) and np.array_equal(g[1], ref[1])
        # the two register-budget variants are compiled separately, so FP32 roundings (FMA
        # contraction) may differ in the last bits
        np.testing.assert_allclose(g[2], ref[2], rtol=1e-6, atol=0)
        np.testing.assert_allclose(g[3], ref[3], atol=1e-5)
    ctx.set_launch(**before)


def test_full_size_forces(workload):
    """Forces of the sampled particles.  WCA on these overpacked workloads spans many
    decades (overlapping pairs), so each row is held to the error its own pairs allow:
    FP64 1e-9 of the row's sum of |U'|; FP32 the change of U' over the FP32 distance
    tolerance plus a 1e-5 turn of each tangent."""
    cfg, mesh, parts, om, src = workload
    face, bary, r_c, pot = cfg["face"], cfg["bary"], cfg["r_c"], cfg["pot"]
    F0, e0 = om.forces_subset(face, bary, r_c, pot, src)
    rows = om.neighbors_gap(face, bary, r_c, sources=src)
    dudl = lambda l: O.pair_dudl(pot, l)
    F, E = css.compute_forces(parts, pot, r_c, css.FP64)
    err = np.linalg.norm(F[src] - F0, axis=1)
    assert np.all(err <= force_row_bounds(rows, pot, dudl, 0.0, FP64_RTOL) + 1e-300)
    tol = FP32_REL_DIAM * synth.bbox_diagonal(cfg["mesh"])
    F32, _ = css.compute_forces(parts, pot, r_c, css.FP32)
    err32 = np.linalg.norm(F32[src] - F0, axis=1)
    assert np.all(err32 <= force_row_bounds(rows, pot, dudl, tol, 1e-5, tie=tol))


def test_hfield_full_size_bd_step():
    """One overdamped step of the whole 8192-particle height-field workload (Philox noise,
    FP64 form) against the oracle's step: identical faces and positions."""
    ctx = css.create(0)
    cfg = synth.make_config("hfield256_n8192")
    m, face, bary, r_c, pot, integ = cfg["mesh"], cfg["face"], cfg["bary"], cfg["r_c"], cfg["pot"], cfg["integ"]
    mesh = css.mesh_upload(ctx, m.verts, m.faces, m.period)
    parts = css.particles_set(ctx, mesh, face, bary, None, None, seed=3)
    css.integrate_step(parts, pot, integ, r_c, css.FP64, 1)
    s = css.particles_get(parts)
    o = O.OracleMesh(m).integrate(face, bary, None, None, None, pot, integ, r_c, 1, seed=3)
    assert np.array_equal(s["face"], o["face"])
    np.testing.assert_allclose(s["bary"], o["bary"], atol=1e-9)
    parts.free()
    mesh.free()
    ctx.close()


def test_noisy_ico8_full_size_abp_step():
    """One active Brownian step of the whole 65536-particle noisy-sphere workload (Philox
    rotational noise, WCA, FP64 form) against the oracle's step: identical faces, positions
    and orientations within 1e-9.  A particle with a pair at a cut-locus tie (two geodesics
    within 1e-12 relative, where the tangent and with it the force direction are set-valued)
    is held only to staying within its displacement cap of the oracle's position."""
    ctx = css.create(0)
    cfg = synth.make_config("noisy_ico8_n65536")
    m, face, bary, r_c, pot, integ = cfg["mesh"], cfg["face"], cfg["bary"], cfg["r_c"], cfg["pot"], cfg["integ"]
    assert integ["kind"] == css.INT_ABP
    mesh = css.mesh_upload(ctx, m.verts, m.faces, m.period)
    parts = css.particles_set(ctx, mesh, face, bary, None, cfg["orient"], seed=5)
    css.integrate_step(parts, pot, integ, r_c, css.FP64, 1)
    s = css.particles_get(parts)
    om = O.OracleMesh(m)
    o = om.integrate(face, bary, None, cfg["orient"], None, pot, integ, r_c, 1, seed=5)
    rows = om.neighbors_gap(face, bary, r_c)
    rs, d, gap = rows[0], rows[2], rows[4]
    tied = np.zeros(len(face), bool)
    for i in np.nonzero(gap <= 1e-12 * np.maximum(d, 1e-300))[0]:
        tied[np.searchsorted(rs, i, side="right") - 1] = True
    assert tied.sum() <= len(face) // 1000
    ok = ~tied
    assert np.array_equal(s["face"][ok], o["face"][ok])
    np.testing.assert_allclose(s["bary"][ok], o["bary"][ok], atol=1e-9)
    np.testing.assert_allclose(s["orient"][ok], o["orient"][ok], atol=1e-9)
    x = synth.particles.world_positions(m, s["face"], s["bary"])
    x0 = synth.particles.world_positions(m, o["face"], o["bary"])
    assert np.all(np.linalg.norm(x - x0, axis=1) <= 2 * integ["max_disp"] + 1e-9)
    parts.free()
    mesh.free()
    ctx.close()


def test_tori64_batched_step():
    """All 64 tori advance one NVE step in one batched launch; sampled sets (smallest,
    median and largest by particle count) equal the oracle's step on that set alone."""
    ctx = css.create(0)
    cfg = synth.make_config("tori64")
    pot, integ, r_c = cfg["pot"], cfg["integ"], cfg["r_c"]
    items = cfg["items"]
    order = np.argsort([len(it["face"]) for it in items], kind="stable")
    check = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    for prec in (css.FP64, css.FP32):
        meshes, sets = [], []
        for it in items:
            mesh = css.mesh_upload(ctx, it["mesh"].verts, it["mesh"].faces)
            meshes.append(mesh)
            sets.append(css.particles_set(ctx, mesh, it["face"], it["bary"], it["vel"]))
        b = css.batch_create(ctx, sets)
        css.batch_step(b, pot, integ, r_c, prec, 1)
        for k in check:
            it = items[k]
            om = O.OracleMesh(it["mesh"])
            F0, _ = om.forces(it["face"], it["bary"], r_c, pot)
            o = om.integrate(it["face"], it["bary"], it["vel"], None, F0, pot, integ, r_c, 1)
            s = css.particles_get(sets[k])
            fscale = max(np.max(np.abs(o["force"])), 1e-300)
            if prec == css.FP64:
                assert np.array_equal(s["face"], o["face"])
                np.testing.assert_allclose(s["bary"], o["bary"], atol=1e-10)
                np.testing.assert_allclose(s["vel"], o["vel"], atol=1e-10)
                assert np.max(np.abs(s["force"] - o["force"])) <= FP64_RTOL * fscale
            else:
                diam = synth.bbox_diagonal(it["mesh"])
                x32 = synth.particles.world_positions(it["mesh"], s["face"], s["bary"])
                x64 = synth.particles.world_positions(it["mesh"], o["face"], o["bary"])
                assert np.max(np.linalg.norm(x32 - x64, axis=1)) <= FP32_REL_DIAM * diam
                # end-of-step forces at the oracle's end positions
                rows = om.neighbors_gap(o["face"], o["bary"], r_c)
                bound = force_row_bounds(rows, pot, lambda l: O.pair_dudl(pot, l), 2 * FP32_REL_DIAM * diam,
                                         1e-5, tie=FP32_REL_DIAM * diam)
                assert np.all(np.linalg.norm(s["force"] - o["force"], axis=1) <= bound)
        b.free()
        for p in sets:
            p.free()
        for mesh in meshes:
            mesh.free()
    ctx.close()


def test_full_size_shortest_paths(workload):
    """Shortest-path polylines (bends included) of every neighbour of three sampled sources
    at full size: the oracle's distance and points (periodic: up to the period), legs
    landing on their nodes, polyline length equal to the distance."""
    cfg, mesh, parts, om, src = workload
    face, bary, r_c = cfg["face"], cfg["bary"], cfg["r_c"]
    s3 = np.sort(src[:3])
    rs, j = om.neighbors(face, bary, r_c, sources=s3)[:2]
    S = np.repeat(s3, np.diff(rs)).astype(np.int32)
    gp, gl, gd, gg = css.geodesic_paths(parts, r_c, S, j, max_points=4096)
    op, ol, od, og = om.geodesic_paths(face, bary, r_c, S, j, cap=4096)
    np.testing.assert_allclose(gd, od, rtol=FP64_RTOL, atol=0)
    per = cfg["mesh"].period
    differ = 0
    for k in range(len(S)):
        assert gg[k] < 1e-9
        dd = np.diff(gp[k], axis=0)
        if per is not None:
            for a in range(2):
                dd[:, a] -= per[a] * np.round(dd[:, a] / per[a])
        assert np.linalg.norm(dd, axis=1).sum() == pytest.approx(gd[k], rel=1e-9)
        # the points decide: a vertex on a straight stretch may end a leg on one side and be
        # passed through mid-leg on the other (equally short chains), which gives the same points
        same = len(gp[k]) == len(op[k])
        if same:
            e = gp[k] - op[k]
            if per is not None:
                for a in range(2):
                    e[:, a] -= per[a] * np.round(e[:, a] / per[a])
            same = bool(np.max(np.abs(e)) < 1e-9)
        differ += not same
    assert differ <= max(1, 0.02 * len(S))
