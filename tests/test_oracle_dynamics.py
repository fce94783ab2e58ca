"""Pins of the CPU oracle's face walk, forces and equations of motion (no GPU)."""
import math

import numpy as np
import pytest

import synth
from oracle import oracle as O
from synth.configs import POT_HARMONIC, POT_WCA, POT_GAUSSIAN, INT_NVE, INT_BD, INT_ABP, INT_GD, INT_FIRE


def _bary_at(m, f, p):
    P = synth.meshes.unwrapped_face_vertices(m)[f]
    M = np.stack([P[1] - P[0], P[2] - P[0]], 1)
    l = np.linalg.lstsq(M, p - P[0], rcond=None)[0]
    return np.array([1 - l.sum(), l[0], l[1]])


def _find(m, p):
    P = synth.meshes.unwrapped_face_vertices(m)
    for f in range(m.nf):
        b = _bary_at(m, f, p)
        if b.min() > -1e-12 and np.linalg.norm(b @ P[f] - p) < 1e-12:
            return f, np.clip(b, 0, None) / np.clip(b, 0, None).sum()
    raise ValueError(p)


# ------------------------------------------------------------------ face walk (Sec. 3.2)
def test_walk_flat_is_vector_addition():
    m = synth.grid_plane(31, 31, -3, 3, -3, 3)
    om = O.OracleMesh(m)
    rng = np.random.default_rng(0)
    for _ in range(50):
        p = np.append(rng.uniform(-1, 1, 2), 0.0)
        d = np.append(rng.uniform(-1.5, 1.5, 2), 0.0)
        v = np.append(rng.normal(size=2), 0.0)
        f, b = _find(m, p)
        f2, b2, cr, nx = om.shift(f, b, d, [v])
        q = om.world([f2], [b2])[0]
        np.testing.assert_allclose(q, p + d, atol=1e-12)
        np.testing.assert_allclose(cr[0], v, atol=1e-12)
        assert nx >= 1 or np.linalg.norm(d) < 0.2


def test_walk_open_boundary_reflects():
    m = synth.grid_plane(11, 11)
    om = O.OracleMesh(m)
    f, b = _find(m, np.array([0.9, 0.53, 0.0]))
    f2, b2, cr, _ = om.shift(f, b, np.array([0.3, 0.1, 0.0]), [np.array([1.0, 2.0, 0.0])])
    np.testing.assert_allclose(om.world([f2], [b2])[0], [0.8, 0.63, 0.0], atol=1e-12)
    np.testing.assert_allclose(cr[0], [-1.0, 2.0, 0.0], atol=1e-12)


def test_walk_around_cube_equator_returns():
    """The band of side faces is flat: a straight walk of length 4 returns unchanged."""
    m = synth.cube(3)
    om = O.OracleMesh(m)
    p = np.array([0.5, 0.0, 0.37])
    f, b = _find(m, p)
    f2, b2, cr, nx = om.shift(f, b, np.array([4.0, 0.0, 0.0]), [np.array([0.3, 0.0, 0.4])])
    np.testing.assert_allclose(om.world([f2], [b2])[0], p, atol=1e-12)
    np.testing.assert_allclose(cr[0], [0.3, 0.0, 0.4], atol=1e-12)
    assert nx >= 12


def test_walk_holonomy_around_cube_corner():
    """Transport around a loop enclosing one cube corner turns vectors by the angle
    defect 2 pi - 3 pi / 2 = pi / 2 (Sec. 3.2: vectors rotate with each edge crossing)."""
    m = synth.cube(2)
    om = O.OracleMesh(m)
    A = np.array([0.75, 0.75, 1.0])
    f, b = _find(m, A)
    v = [np.array([1.0, 0.0, 0.0])]
    f, b, v, _ = om.shift(f, b, np.array([0.5, 0.0, 0.0]), v)       # top -> x=1 side
    np.testing.assert_allclose(om.world([f], [b])[0], [1.0, 0.75, 0.75], atol=1e-12)
    f, b, v, _ = om.shift(f, b, np.array([0.0, 0.5, 0.0]), v)       # x=1 -> y=1 side
    np.testing.assert_allclose(om.world([f], [b])[0], [0.75, 1.0, 0.75], atol=1e-12)
    f, b, v, _ = om.shift(f, b, np.array([0.0, 0.0, 0.5]), v)       # y=1 side -> top
    np.testing.assert_allclose(om.world([f], [b])[0], A, atol=1e-12)
    np.testing.assert_allclose(v[0], [0.0, 1.0, 0.0], atol=1e-12)


def test_walk_tube_is_unrolled_line():
    """Developable tube: a walk is a straight line of the unrolled strip (wrapping around)."""
    n = 10
    m = synth.cylinder_tube(n, 4, 1.0, 4.0)
    om = O.OracleMesh(m)
    side = 2 * math.sin(math.pi / n)
    P = n * side
    corner = lambda k: np.array([math.cos(2 * math.pi * k / n), math.sin(2 * math.pi * k / n)])
    e0 = np.append((corner(1) - corner(0)) / side, 0.0)
    u0, z0 = 0.3 * side, 1.013
    start = np.append(corner(0), z0) + u0 * e0
    f, b = _find(m, start)
    du, dz = 1.7 * P, 0.9
    f2, b2, _, nx = om.shift(f, b, du * e0 + dz * np.array([0.0, 0.0, 1.0]), None)
    u_end = (u0 + du) % P
    k = int(u_end // side)
    xy = corner(k) + (u_end - k * side) * (corner(k + 1) - corner(k)) / side
    np.testing.assert_allclose(om.world([f2], [b2])[0], [xy[0], xy[1], z0 + dz], atol=1e-11)
    assert nx > 17


def test_walk_preserves_length_and_reverses():
    m = synth.icosphere(3, 1.0, noise=0.02, seed=4)
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 30, 3)
    dirs = synth.random_tangent_units(m, face, 5)
    carry = synth.random_tangent_units(m, face, 6)
    for i in range(30):
        d = 0.4 * dirs[i]
        f2, b2, cr, _ = om.shift(face[i], bary[i], d, [d, carry[i]])
        np.testing.assert_allclose(np.linalg.norm(cr, axis=1), [0.4, 1.0], rtol=1e-13)
        fr = om.face_frame(f2)
        nrm = np.cross(fr[1], fr[2])
        assert abs(cr[0] @ nrm) < 1e-13 and abs(cr[1] @ nrm) < 1e-13
        f3, b3, cr2, _ = om.shift(f2, b2, -cr[0], [cr[1]])
        np.testing.assert_allclose(om.world([f3], [b3])[0], om.world([face[i]], [bary[i]])[0], atol=1e-12)
        np.testing.assert_allclose(cr2[0], carry[i], atol=1e-12)


# ------------------------------------------------------------------ forces (Sec. 2.1, Sec. 3.1)
def test_pair_potentials_closed_forms():
    h = dict(kind=POT_HARMONIC, eps=1.0, sigma=0.1, r_cut=0.1, A=1.0)
    assert O.pair_energy(h, 0.05) == pytest.approx(0.25)
    assert O.pair_dudl(h, 0.05) == pytest.approx(-10.0)
    assert O.pair_energy(h, 0.1) == 0.0
    s = 0.2
    w = dict(kind=POT_WCA, eps=1.0, sigma=s, r_cut=2 ** (1 / 6) * s, A=1.0)
    assert O.pair_energy(w, 2 ** (1 / 6) * s * (1 - 1e-12)) == pytest.approx(0.0, abs=1e-9)
    assert O.pair_energy(w, s) == pytest.approx(1.0)
    assert O.pair_dudl(w, s) == pytest.approx(-24.0 / s)
    g = dict(kind=POT_GAUSSIAN, eps=1.0, sigma=0.5, r_cut=10.0, A=2.0)
    l = 0.3
    assert O.pair_energy(g, l) == pytest.approx(2.0 * math.exp(-l * l / 0.5))
    # the paper's f = (l / sigma^2) U grad l  <=>  dU/dl = -(l / sigma^2) U
    assert O.pair_dudl(g, l) == pytest.approx(-(l / 0.25) * O.pair_energy(g, l))


def test_flat_forces_equal_euclidean():
    cfg = synth.make_config("flat64")
    m, face, bary, pot = cfg["mesh"], cfg["face"], cfg["bary"], cfg["pot"]
    om = O.OracleMesh(m)
    F, E = om.forces(face, bary, math.inf, pot)
    x = synth.particles.world_positions(m, face, bary)
    Fw = np.zeros_like(x)
    Ew = 0.0
    s = pot["sigma"]
    for i in range(len(x)):
        for j in range(len(x)):
            if i == j:
                continue
            dx = x[j] - x[i]
            r = np.linalg.norm(dx)
            if r < s:
                Fw[i] += -2 * (1 - r / s) / s * dx / r
                Ew += 0.5 * (1 - r / s) ** 2
    np.testing.assert_allclose(F, Fw, atol=1e-12)
    assert E == pytest.approx(Ew, rel=1e-12)


def test_subset_forces_equal_euclidean_rows():
    """Forces on a listed subset follow the same flat closed form; the per-particle half
    energies add up to the total."""
    cfg = synth.make_config("flat64")
    m, face, bary, pot = cfg["mesh"], cfg["face"], cfg["bary"], cfg["pot"]
    om = O.OracleMesh(m)
    x = synth.particles.world_positions(m, face, bary)
    src = [5, 0, 63, 17]
    F, e = om.forces_subset(face, bary, math.inf, pot, src)
    s = pot["sigma"]
    for k, i in enumerate(src):
        Fw = np.zeros(3)
        ew = 0.0
        for j in range(len(x)):
            r = np.linalg.norm(x[j] - x[i])
            if j != i and r < s:
                Fw += -2 * (1 - r / s) / s * (x[j] - x[i]) / r
                ew += 0.5 * (1 - r / s) ** 2
        np.testing.assert_allclose(F[k], Fw, atol=1e-12)
        assert e[k] == pytest.approx(ew, rel=1e-12, abs=1e-15)
    _, e_all = om.forces_subset(face, bary, math.inf, pot, np.arange(len(face)))
    _, E = om.forces(face, bary, math.inf, pot)
    assert e_all.sum() == pytest.approx(E, rel=1e-12)


def test_forces_are_minus_energy_gradient():
    """F_i = -dE/dx_i along the tangent plane, by central differences on a curved mesh."""
    m = synth.icosphere(3, 1.0, noise=0.01, seed=1)
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 40, 2)
    pot = dict(kind=POT_GAUSSIAN, eps=1.0, sigma=0.25, r_cut=0.9, A=1.0)
    F, E0 = om.forces(face, bary, 0.9, pot)
    eps = 1e-5
    u = synth.random_tangent_units(m, face, 3)
    checked = 0
    for i in range(0, 40, 4):
        E = []
        for sgn in (1, -1):
            f2, b2, _, nx = om.shift(face[i], bary[i], sgn * eps * u[i], None)
            fc, bc = face.copy(), bary.copy()
            fc[i], bc[i] = f2, b2
            E.append(om.forces(fc, bc, 0.9, pot)[1])
        dEdu = (E[0] - E[1]) / (2 * eps)
        assert dEdu == pytest.approx(-F[i] @ u[i], abs=2e-6 * (1 + abs(dEdu)))
        checked += 1
    assert checked == 10


# ------------------------------------------------------------------ dynamics (Sec. 2.1)
def _nve_drift(om, m, face, bary, vel, pot, dt, T, rc):
    integ = dict(kind=INT_NVE, dt=dt, kT=0.0, lam=1.0, v0=0.0, Dr=0.0, mass=1.0, max_disp=math.inf)
    F, E = om.forces(face, bary, rc, pot)
    s = dict(face=face, bary=bary, vel=vel, force=F, epot=E)
    e0 = E + 0.5 * np.sum(vel ** 2)
    drift = 0.0
    for _ in range(int(round(T / dt))):
        s = om.integrate(s["face"], s["bary"], s["vel"], None, s["force"], pot, integ, rc, 1)
        e = s["epot"] + 0.5 * np.sum(s["vel"] ** 2)
        drift = max(drift, abs(e - e0))
    return drift


def test_nve_energy_error_is_second_order():
    """Velocity Verlet (Sec. 2.1): energy error ~ dt^2 where distances are smooth (flat
    periodic patch, Gaussian truncated where U ~ 1e-7)."""
    m = synth.periodic_heightfield(16, 1, seed=0, A=(0.0, 0.0))
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 40, 6)
    vel = synth.gaussian_tangent_velocities(m, face, 0.5, 1.0, 7)
    pot = dict(kind=POT_GAUSSIAN, eps=1.0, sigma=0.08, r_cut=0.45, A=1.0)
    d1 = _nve_drift(om, m, face, bary, vel, pot, 0.004, 0.2, 0.45)
    d2 = _nve_drift(om, m, face, bary, vel, pot, 0.002, 0.2, 0.45)
    assert d1 > 0
    assert 3.2 < d1 / d2 < 4.8


def test_nve_conserves_energy_on_curved_mesh():
    m = synth.icosphere(3, 1.0)
    om = O.OracleMesh(m)
    face, bary = synth.place_uniform(m, 24, 6)
    vel = synth.gaussian_tangent_velocities(m, face, 0.5, 1.0, 7)
    pot = dict(kind=POT_HARMONIC, eps=1.0, sigma=0.4, r_cut=0.4, A=1.0)
    F, E = om.forces(face, bary, 0.4, pot)
    e0 = E + 0.5 * np.sum(vel ** 2)
    d = _nve_drift(om, m, face, bary, vel, pot, 0.005, 0.5, 0.4)
    assert d < 2e-3 * e0


def test_bd_injected_noise_step_is_exact():
    m = synth.grid_plane(11, 11, -2, 2, -2, 2)
    om = O.OracleMesh(m)
    f, b = _find(m, np.array([0.1, 0.2, 0.0]))
    pot = dict(kind=POT_HARMONIC, eps=0.0, sigma=0.1, r_cut=0.1, A=1.0)
    integ = dict(kind=INT_BD, dt=1e-3, kT=2.0, lam=0.5, v0=0.0, Dr=0.0, mass=1.0, max_disp=math.inf)
    noise = np.array([[0.7, -1.3]])
    s = om.integrate([f], [b], None, None, None, pot, integ, 0.1, 1, noise=noise)
    amp = math.sqrt(2 * 2.0 * 1e-3 / 0.5)
    fr = om.face_frame(f)
    want = np.array([0.1, 0.2, 0.0]) + amp * (0.7 * fr[1] - 1.3 * fr[2])
    np.testing.assert_allclose(om.world(s["face"], s["bary"])[0], want, atol=1e-13)


def test_bd_free_diffusion_msd():
    """<|dr|^2> = 4 kT t / lambda for free 2D Brownian motion on a flat patch."""
    m = synth.grid_plane(21, 21, -5, 5, -5, 5)
    om = O.OracleMesh(m)
    n = 3000
    rng = np.random.default_rng(1)
    pts = np.concatenate([rng.uniform(-0.5, 0.5, (n, 2)), np.zeros((n, 1))], 1)
    fb = [_find(m, p) for p in pts[:200]]
    face = np.array([f for f, _ in fb] * 15, np.int32)
    bary = np.array([b for _, b in fb] * 15)
    x0 = om.world(face, bary)
    pot = dict(kind=POT_HARMONIC, eps=0.0, sigma=1e-3, r_cut=1e-3, A=1.0)
    integ = dict(kind=INT_BD, dt=0.01, kT=1.0, lam=1.0, v0=0.0, Dr=0.0, mass=1.0, max_disp=math.inf)
    s = om.integrate(face, bary, None, None, None, pot, integ, 1e-3, 10, seed=123)
    msd = np.mean(np.sum((om.world(s["face"], s["bary"]) - x0) ** 2, axis=1))
    assert msd == pytest.approx(4 * 1.0 * 0.1, rel=0.06)


def test_abp_self_propulsion_and_rotation():
    m = synth.grid_plane(11, 11, -2, 2, -2, 2)
    om = O.OracleMesh(m)
    f, b = _find(m, np.array([0.1, 0.2, 0.0]))
    pot = dict(kind=POT_HARMONIC, eps=0.0, sigma=1e-3, r_cut=1e-3, A=1.0)
    integ = dict(kind=INT_ABP, dt=0.01, kT=0.0, lam=1.0, v0=1.5, Dr=0.2, mass=1.0, max_disp=math.inf)
    n0 = np.array([[0.6, 0.8, 0.0]])
    z = 0.9
    s = om.integrate([f], [b], None, n0, None, pot, integ, 1e-3, 1, noise=np.array([[z, 0.0]]))
    np.testing.assert_allclose(om.world(s["face"], s["bary"])[0], [0.1 + 0.015 * 0.6, 0.2 + 0.015 * 0.8, 0], atol=1e-13)
    a = math.sqrt(2 * 0.2 * 0.01) * z
    want = np.array([0.6 * math.cos(a) - 0.8 * math.sin(a), 0.6 * math.sin(a) + 0.8 * math.cos(a), 0.0])
    np.testing.assert_allclose(s["orient"][0], want, atol=1e-13)


def test_displacement_clamp():
    m = synth.grid_plane(11, 11, -2, 2, -2, 2)
    om = O.OracleMesh(m)
    f, b = _find(m, np.array([0.1, 0.2, 0.0]))
    pot = dict(kind=POT_HARMONIC, eps=0.0, sigma=1e-3, r_cut=1e-3, A=1.0)
    integ = dict(kind=INT_ABP, dt=1.0, kT=0.0, lam=1.0, v0=5.0, Dr=0.0, mass=1.0, max_disp=0.25)
    s = om.integrate([f], [b], None, np.array([[1.0, 0.0, 0.0]]), None, pot, integ, 1e-3, 1,
                     noise=np.zeros((1, 2)))
    np.testing.assert_allclose(om.world(s["face"], s["bary"])[0], [0.35, 0.2, 0.0], atol=1e-13)


# ------------------------------------------------------------------ minimisers (Fig. 3)
def _pair_on_plane(d):
    m = synth.grid_plane(31, 31, -3, 3, -3, 3)
    locs = [_find(m, np.array([-d / 2, 0.013, 0.0])), _find(m, np.array([d / 2, 0.013, 0.0]))]
    face = np.array([f for f, _ in locs], np.int32)
    bary = np.array([b for _, b in locs])
    return m, face, bary


def test_steepest_descent_step_closed_form():
    """One descent step of two harmonic particles on a plane moves each away from the
    other by (dt / lambda) |U'(d)|: d' = d + 2 (dt / lambda) 2 (1 - d / sigma) / sigma."""
    d, sig, dt, lam = 0.3, 0.5, 0.01, 2.0
    m, face, bary = _pair_on_plane(d)
    om = O.OracleMesh(m)
    pot = dict(kind=POT_HARMONIC, eps=1.0, sigma=sig, r_cut=sig)
    integ = dict(kind=INT_GD, dt=dt, kT=5.0, lam=lam, v0=0.0, Dr=0.0, mass=1.0, max_disp=1.0)
    o = om.integrate(face, bary, None, None, None, pot, integ, math.inf, 1)
    x = om.world(o["face"], o["bary"])
    expect = d + 2 * (dt / lam) * 2 * (1 - d / sig) / sig
    assert np.linalg.norm(x[1] - x[0]) == pytest.approx(expect, rel=1e-12)
    # kT is ignored: descent draws no noise
    o2 = om.integrate(face, bary, None, None, None, pot, dict(integ, kT=0.0), math.inf, 1)
    np.testing.assert_array_equal(o["bary"], o2["bary"])


def test_fire_first_steps_closed_form():
    """FIRE from rest: P = 0 halves dt and keeps v = 0, so the first step is a velocity-Verlet
    step of dt/2 from rest (each particle moves (dt/2)^2/2 |F| / m); on the second step v is
    parallel to F (P > 0, the mixing leaves it unchanged, dt unchanged before N_min)."""
    d, sig, dt = 0.3, 0.5, 0.02
    m, face, bary = _pair_on_plane(d)
    om = O.OracleMesh(m)
    pot = dict(kind=POT_HARMONIC, eps=1.0, sigma=sig, r_cut=sig)
    integ = dict(kind=INT_FIRE, dt=dt, kT=0.0, lam=1.0, v0=0.0, Dr=0.0, mass=1.0, max_disp=1.0)
    F0, _ = om.forces(face, bary, math.inf, pot)
    o = om.fire(face, bary, None, F0, pot, integ, math.inf, 1)
    fmag = 2 * (1 - d / sig) / sig
    h = dt / 2
    d1 = d + 2 * 0.5 * h * h * fmag
    x = om.world(o["face"], o["bary"])
    assert np.linalg.norm(x[1] - x[0]) == pytest.approx(d1, rel=1e-12)
    np.testing.assert_allclose(o["state"], [dt / 2, 0.1, 0.0])
    f1 = 2 * (1 - d1 / sig) / sig
    assert np.linalg.norm(o["vel"][0]) == pytest.approx(0.5 * h * (fmag + f1), rel=1e-12)
    o2 = om.fire(o["face"], o["bary"], o["vel"], o["force"], pot, integ, math.inf, 1, state=o["state"])
    np.testing.assert_allclose(o2["state"], [dt / 2, 0.1, 1.0])
    v1 = 0.5 * h * (fmag + f1)
    d2 = d1 + 2 * (h * (v1 + 0.5 * h * f1))
    x2 = om.world(o2["face"], o2["bary"])
    assert np.linalg.norm(x2[1] - x2[0]) == pytest.approx(d2, rel=1e-12)


def test_fire_relaxes_a_dilute_repulsive_system():
    """Particles on a torus with soft repulsion relax to zero force (all pairs pushed apart
    beyond the range): the energy ends far below its start and the forces vanish."""
    m = synth.torus(3.0, 1.0, 48, 16)
    face, bary = synth.place_uniform(m, 40, 3)
    om = O.OracleMesh(m)
    pot = dict(kind=POT_HARMONIC, eps=1.0, sigma=0.6, r_cut=0.6)
    integ = dict(kind=INT_FIRE, dt=0.02, kT=0.0, lam=1.0, v0=0.0, Dr=0.0, mass=1.0, max_disp=0.1)
    F0, E0 = om.forces(face, bary, 0.6, pot)
    o = om.fire(face, bary, None, F0, pot, integ, 0.6, 400)
    assert E0 > 0.1
    assert o["epot"] < 1e-6 * E0
    assert np.max(np.abs(o["force"])) < 1e-3
