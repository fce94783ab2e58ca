"""The five benchmark workloads as seeded synthetic inputs.

Each builder returns a dict with the mesh(es), the particle state and the
potential / integrator parameters.  Where the workload statement is silent a
documented reading is used (listed next to each field).
"""
from __future__ import annotations

import math

import numpy as np

from .meshes import grid_plane, icosphere, periodic_heightfield, torus
from .particles import place_uniform, gaussian_tangent_velocities, random_tangent_units

CONFIG_NAMES = ("flat64", "ico5_n1024", "hfield256_n8192", "tori64", "noisy_ico8_n65536")

# potential kinds, shared numbering with the C ABI header and the oracle
POT_HARMONIC, POT_WCA, POT_GAUSSIAN = 0, 1, 2
# integrator kinds
INT_NVE, INT_BD, INT_ABP, INT_GD, INT_FIRE = 0, 1, 2, 3, 4

WCA_RCUT = 2.0 ** (1.0 / 6.0)


def _flat64(seed=1, n=64):
    m = grid_plane(21, 21)
    face, bary = place_uniform(m, n, seed, area_weighted=False)
    vel = gaussian_tangent_velocities(m, face, kT=0.1, mass=1.0, seed=seed + 100)
    return dict(name="flat64", mesh=m, face=face, bary=bary, vel=vel, orient=None,
                r_c=math.inf,
                pot=dict(kind=POT_HARMONIC, eps=1.0, sigma=0.1, r_cut=0.1, A=1.0),
                integ=dict(kind=INT_NVE, dt=0.005, kT=0.1, lam=1.0, v0=0.0, Dr=0.0,
                           mass=1.0, max_disp=math.inf),
                steps=10)


def _ico5(seed=2, n=1024):
    m = icosphere(5, 1.0)
    face, bary = place_uniform(m, n, seed)
    # reading: initial velocities as in the flat workload, N(0, 0.1) per component
    vel = gaussian_tangent_velocities(m, face, kT=0.1, mass=1.0, seed=seed + 100)
    return dict(name="ico5_n1024", mesh=m, face=face, bary=bary, vel=vel, orient=None,
                r_c=0.15,
                pot=dict(kind=POT_HARMONIC, eps=1.0, sigma=0.15, r_cut=0.15, A=1.0),
                integ=dict(kind=INT_NVE, dt=0.002, kT=0.1, lam=1.0, v0=0.0, Dr=0.0,
                           mass=1.0, max_disp=math.inf),
                steps=1000)


def _hfield(seed=3, n=8192, grid=256):
    m = periodic_heightfield(grid, 32, seed)
    face, bary = place_uniform(m, n, seed + 10)
    r_c = 0.05
    sigma = r_c / WCA_RCUT          # reading: WCA cut at r_c = 2^(1/6) sigma
    return dict(name="hfield256_n8192", mesh=m, face=face, bary=bary, vel=None, orient=None,
                r_c=r_c,
                pot=dict(kind=POT_WCA, eps=1.0, sigma=sigma, r_cut=r_c, A=1.0),
                # readings: lambda = kT = 1, dt = 1e-5, displacement clamp 0.5 r_c
                integ=dict(kind=INT_BD, dt=1e-5, kT=1.0, lam=1.0, v0=0.0, Dr=0.0,
                           mass=1.0, max_disp=0.5 * r_c),
                steps=500)


def torus_for_faces(F_target: int, R: float, r: float):
    n_v = max(3, int(round(math.sqrt(F_target / 2.0 * r / R))))
    n_u = max(3, int(round(F_target / (2.0 * n_v))))
    return torus(R, r, n_u, n_v)


def _tori(seed=4, n_mesh=64, f_lo=2000, f_hi=60000, n_lo=128, n_hi=4096):
    rng = np.random.default_rng(seed)
    items = []
    for k in range(n_mesh):
        R = rng.uniform(1.0, 3.0)
        r = rng.uniform(0.3, 0.9)
        F = int(round(math.exp(rng.uniform(math.log(f_lo), math.log(f_hi)))))
        N = int(rng.integers(n_lo, n_hi + 1))
        m = torus_for_faces(F, R, r)
        face, bary = place_uniform(m, N, 4000 + k)
        vel = gaussian_tangent_velocities(m, face, kT=0.1, mass=1.0, seed=5000 + k)
        items.append(dict(mesh=m, face=face, bary=bary, vel=vel))
    return dict(name="tori64", items=items, r_c=0.1,
                pot=dict(kind=POT_HARMONIC, eps=1.0, sigma=0.1, r_cut=0.1, A=1.0),
                # reading: dt as in the icosphere workload
                integ=dict(kind=INT_NVE, dt=0.002, kT=0.1, lam=1.0, v0=0.0, Dr=0.0,
                           mass=1.0, max_disp=math.inf),
                steps=200)


def _noisy_ico8(seed=5, n=65536, level=8):
    m = icosphere(level, 10.0, noise=0.02, seed=seed)
    face, bary = place_uniform(m, n, seed + 10)
    orient = random_tangent_units(m, face, seed + 20)
    sigma = 0.2
    r_c = WCA_RCUT * sigma
    return dict(name="noisy_ico8_n65536", mesh=m, face=face, bary=bary, vel=None,
                orient=orient, r_c=r_c,
                pot=dict(kind=POT_WCA, eps=1.0, sigma=sigma, r_cut=r_c, A=1.0),
                # readings: unit mobility, no translational noise, clamp 0.5 r_c
                integ=dict(kind=INT_ABP, dt=1e-3, kT=0.0, lam=1.0, v0=1.0, Dr=0.1,
                           mass=1.0, max_disp=0.5 * r_c),
                steps=1000)


def make_config(name: str, **kw):
    builders = {"flat64": _flat64, "ico5_n1024": _ico5, "hfield256_n8192": _hfield,
                "tori64": _tori, "noisy_ico8_n65536": _noisy_ico8}
    return builders[name](**kw)
