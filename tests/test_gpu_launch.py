"""Launch shapes, the two-pass deferral and the autotuner (needs a GB300).

The result of a neighbour / force evaluation must not depend on how it is launched:
every shape below -- shared-memory tables of each scale or global tables, 1 to 8 warps
per CTA, capped residency, tiled work claims, and first-pass pools so small that most
sources overflow and are re-run by the second pass -- gives the same neighbour rows, with
distances equal to 1e-14 relative and FP64 forces equal up to summation order, and they
match the oracle.
"""
import numpy as np
import pytest

import synth
from oracle import oracle as O
from tests._common import FP64_RTOL, compare_pairs

css = pytest.importorskip("paper_2404_19751_gb300")
pytestmark = pytest.mark.gpu

BASE = dict(warps_per_cta=4, ctas_per_sm=0, tile=1, shared_scale=1, window_capacity=2048,
            window_capacity2=16384, warps2_per_sm=2, occupancy=1, table_capacity=0, team=0)

SHAPES = [
    dict(),
    dict(shared_scale=0),
    dict(shared_scale=2, warps_per_cta=2),
    dict(shared_scale=4, warps_per_cta=2, ctas_per_sm=1),
    dict(warps_per_cta=1, tile=4),
    dict(warps_per_cta=8, tile=16),
    dict(window_capacity=64, window_capacity2=128),        # nearly every source deferred
    dict(shared_scale=1, window_capacity=256, warps2_per_sm=1),
    dict(occupancy=2, warps_per_cta=8),
    dict(occupancy=2, shared_scale=0, window_capacity=8192, tile=2),
    dict(shared_scale=0, window_capacity=8192, table_capacity=256),    # small tables: some deferred
    dict(occupancy=2, shared_scale=0, window_capacity=32768, table_capacity=2048, warps_per_cta=8),
    # team form: all warps of a CTA on one source
    dict(team=1, warps_per_cta=2),
    dict(team=1, warps_per_cta=8, shared_scale=0, window_capacity=8192),
    dict(team=1, warps_per_cta=4, occupancy=2, shared_scale=0, window_capacity=8192),
    dict(team=1, warps_per_cta=4, window_capacity=64, window_capacity2=128),   # most sources deferred
]


@pytest.fixture(scope="module")
def case():
    m = synth.icosphere(4, 1.0, noise=0.015, seed=4)
    face, bary = synth.place_uniform(m, 1500, 6)
    r_c = 0.3
    pot = dict(kind=css.POT_HARMONIC, eps=1.0, sigma=r_c, r_cut=r_c)
    om = O.OracleMesh(m)
    F0, E0 = om.forces(face, bary, r_c, pot)
    rows = om.neighbors_gap(face, bary, r_c)
    return m, face, bary, r_c, pot, F0, E0, rows


def test_results_do_not_depend_on_launch_shape(case):
    m, face, bary, r_c, pot, F0, E0, rows = case
    ctx = css.create(0)
    mesh = css.mesh_upload(ctx, m.verts, m.faces)
    parts = css.particles_set(ctx, mesh, face, bary)
    ref = None
    deferred = []
    for sh in SHAPES:
        ctx.set_launch(**dict(BASE, **sh))
        F, E = css.compute_forces(parts, pot, r_c, css.FP64)
        deferred.append(ctx.last_counters()["deferred"])
        assert ctx.last_counters()["sources"] == len(face)
        assert np.max(np.abs(F - F0)) <= FP64_RTOL * np.max(np.abs(F0)), sh
        assert E == pytest.approx(E0, rel=1e-10)
        g = css.geodesic_neighbors(parts, r_c, css.FP64)
        compare_pairs(g, rows, r_c, FP64_RTOL, 1e-7)
        if ref is None:
            ref = (F, g)
        else:
            # the pair set is the same in every shape.  The pool slot (and queue position) a
            # window gets depends on the order in which diverging lanes of one insertion round
            # reach their allocation, which the table placement's latencies change; a team
            # unfolds wider waves.  Either way a distance that two equally long unfoldings
            # reach (a vertex lying exactly on a straight path, say) may take the other's last
            # bit, and a row's force sum may run in another order
            assert np.max(np.abs(F - ref[0])) <= 1e-13 * np.max(np.abs(F0)), sh
            assert np.array_equal(g[0], ref[1][0]) and np.array_equal(g[1], ref[1][1])
            np.testing.assert_allclose(g[2], ref[1][2], rtol=1e-14, atol=0)
    assert deferred[0] == 0 and deferred[6] > len(face) // 2   # the tiny pool defers most sources
    assert deferred[10] > 0                                    # so do tables of 256 edge slots
    assert deferred[15] > len(face) // 2                       # and a team's tiny pool
    parts.free()
    mesh.free()
    ctx.close()


def test_launch_shape_validation():
    ctx = css.create(0)
    for bad in (dict(warps_per_cta=0), dict(warps_per_cta=9), dict(shared_scale=3), dict(tile=0),
                dict(window_capacity=10), dict(warps2_per_sm=0), dict(shared_scale=8, warps_per_cta=8),
                dict(occupancy=3), dict(table_capacity=10), dict(table_capacity=1 << 21),
                dict(team=1, warps_per_cta=1), dict(team=2)):
        with pytest.raises(css.CssError):
            ctx.set_launch(**dict(BASE, **bad))
    assert ctx.get_launch() == dict(BASE)    # a rejected shape leaves the old one
    ctx.close()


def test_autotuner_keeps_results_and_state(case):
    m, face, bary, r_c, pot, F0, E0, rows = case
    ctx = css.create(0)
    mesh = css.mesh_upload(ctx, m.verts, m.faces)
    parts = css.particles_set(ctx, mesh, face, bary)
    before = css.particles_get(parts)
    shape, ms = ctx.autotune([parts], pot, r_c, css.FP32, reps=1, sample=600)
    assert ms > 0 and shape == ctx.get_launch()
    after = css.particles_get(parts)
    assert np.array_equal(before["face"], after["face"]) and np.array_equal(before["bary"], after["bary"])
    F, E = css.compute_forces(parts, pot, r_c, css.FP64)
    assert np.max(np.abs(F - F0)) <= FP64_RTOL * np.max(np.abs(F0))
    parts.free()
    mesh.free()
    ctx.close()


def test_autotuner_on_a_batch_then_batched_steps_match_single_sets():
    """The tuner times one launch over all sets of a batch; the batched steps that follow
    in the tuned shape equal the same sets stepped alone in the default shape."""
    ctx = css.create(0)
    pot = dict(kind=css.POT_HARMONIC, eps=1.0, sigma=0.1, r_cut=0.1)
    integ = dict(kind=css.INT_NVE, dt=0.002, kT=0.1, lam=1.0, v0=0.0, Dr=0.0, mass=1.0, max_disp=float("inf"))
    meshes, sets, states = [], [], []
    for k in range(4):
        m = synth.configs.torus_for_faces(2500 + 2000 * k, 2.0 + 0.2 * k, 0.4 + 0.1 * k)
        face, bary = synth.place_uniform(m, 300 + 150 * k, 80 + k)
        vel = synth.gaussian_tangent_velocities(m, face, 0.1, 1.0, 90 + k)
        mesh = css.mesh_upload(ctx, m.verts, m.faces)
        meshes.append(mesh)
        sets.append(css.particles_set(ctx, mesh, face, bary, vel))
        states.append((face, bary, vel))
    ctx.set_launch(**BASE)
    singles = [css.particles_set(ctx, mh, *st) for mh, st in zip(meshes, states)]
    for p in singles:
        css.integrate_step(p, pot, integ, 0.1, css.FP64, 4)
    shape, ms = ctx.autotune(sets, pot, 0.1, css.FP64, reps=1, sample=500)
    assert ms > 0 and shape == ctx.get_launch()
    b = css.batch_create(ctx, sets)
    css.batch_step(b, pot, integ, 0.1, css.FP64, 4)
    for pb, ps in zip(sets, singles):
        a, c = css.particles_get(pb), css.particles_get(ps)
        assert np.array_equal(a["face"], c["face"])
        np.testing.assert_allclose(a["bary"], c["bary"], atol=1e-12)
        np.testing.assert_allclose(a["vel"], c["vel"], atol=1e-12)
    b.free()
    for p in sets + singles:
        p.free()
    for mh in meshes:
        mh.free()
    ctx.close()


@pytest.mark.parametrize("name", ["flat64", "saddle_fan8_n40"])
def test_team_form_matches_oracle(name):
    """The team form on all-pairs workloads with few sources (the flat plane's 64, a saddle
    cone's 40): FP64 neighbours and forces equal the oracle's, FP32 within its bar, and an
    NVE step equals the oracle's step."""
    from tests.test_gpu_parity import WORKLOADS
    from tests._common import FP32_REL_DIAM, descent_checker
    import math
    m, face, bary, r_c = WORKLOADS[name]()
    sig = 0.3
    pot = dict(kind=css.POT_HARMONIC, eps=1.0, sigma=sig, r_cut=sig)
    ctx = css.create(0)
    mesh = css.mesh_upload(ctx, m.verts, m.faces, m.period)
    om = O.OracleMesh(m)
    rows = om.neighbors_gap(face, bary, r_c)
    F0, E0 = om.forces(face, bary, sig, pot)
    for sh in (dict(team=1, warps_per_cta=8), dict(team=1, warps_per_cta=4, shared_scale=0, window_capacity=8192)):
        ctx.set_launch(**dict(BASE, **sh))
        parts = css.particles_set(ctx, mesh, face, bary)
        g = css.geodesic_neighbors(parts, r_c, css.FP64)
        compare_pairs(g, rows, r_c, FP64_RTOL, 1e-7)
        F, E = css.compute_forces(parts, pot, sig, css.FP64)
        assert np.max(np.abs(F - F0)) <= FP64_RTOL * np.max(np.abs(F0))
        assert E == pytest.approx(E0, rel=1e-10)
        tol = FP32_REL_DIAM * synth.bbox_diagonal(m)
        g32 = css.geodesic_neighbors(parts, r_c, css.FP32)
        compare_pairs(g32, rows, r_c, tol, 1e-5, rel=False, band=tol, tie=tol,
                      walker=descent_checker(om, face, bary, r_c), land_tol=1e-7)
        parts.free()
    vel = synth.gaussian_tangent_velocities(m, face, 0.1, 1.0, 5)
    integ = dict(kind=css.INT_NVE, dt=0.002, kT=0.1, lam=1.0, v0=0.0, Dr=0.0, mass=1.0, max_disp=math.inf)
    parts = css.particles_set(ctx, mesh, face, bary, vel)
    css.integrate_step(parts, pot, integ, sig, css.FP64, 2)
    s = css.particles_get(parts)
    o = om.integrate(face, bary, vel, None, F0, pot, integ, sig, 2)
    assert np.array_equal(s["face"], o["face"])
    np.testing.assert_allclose(s["bary"], o["bary"], atol=1e-9)
    parts.free()
    mesh.free()
    ctx.close()
