"""ctypes wrapper around the C oracle (TEST INFRASTRUCTURE ONLY)."""
from __future__ import annotations

import ctypes as C
import math
from typing import Optional

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.om_mesh_create.argtypes = [P, C.c_int64, P, C.c_int64, P, C.POINTER(C.c_void_p)]
        L.om_mesh_create.restype = C.c_int
        L.om_mesh_destroy.argtypes = [P]
        L.om_mesh_num_edges.argtypes = [P]
        L.om_mesh_num_edges.restype = C.c_int64
        L.om_mesh_vertex_info.argtypes = [P, P, P, P]
        L.om_face_frame.argtypes = [P, C.c_int32, P]
        L.om_world_position.argtypes = [P, C.c_int32, P, P]
        L.om_geodesic_query.argtypes = [P, C.c_int32, P, C.c_double, C.c_int64, P, P, P, P, P]
        L.om_geodesic_query.restype = C.c_int
        L.om_neighbors.argtypes = [P, C.c_int64, P, P, C.c_double, C.c_int64, P, P, P, P, P, C.c_int, P]
        L.om_neighbors.restype = C.c_int
        L.om_neighbors_subset.argtypes = [P, C.c_int64, P, P, C.c_double, C.c_int64, P, C.c_int64,
                                          P, P, P, P, P, C.c_int, P]
        L.om_neighbors_subset.restype = C.c_int
        L.om_neighbors_gap.argtypes = [P, C.c_int64, P, P, C.c_double, C.c_int64, P, C.c_int64,
                                       P, P, P, P, P, P, C.c_int, P]
        L.om_neighbors_gap.restype = C.c_int
        L.om_pair_energy.argtypes = [P, C.c_double]
        L.om_pair_energy.restype = C.c_double
        L.om_pair_dudl.argtypes = [P, C.c_double]
        L.om_pair_dudl.restype = C.c_double
        L.om_forces.argtypes = [P, C.c_int64, P, P, C.c_double, P, P, P, C.c_int]
        L.om_forces.restype = C.c_int
        L.om_forces_subset.argtypes = [P, C.c_int64, P, P, C.c_double, P, C.c_int64, P, P, P, C.c_int]
        L.om_forces_subset.restype = C.c_int
        L.om_shift.argtypes = [P, P, P, P, C.c_int, P]
        L.om_shift.restype = C.c_int
        L.om_integrate.argtypes = [P, C.c_int64, P, P, P, P, P, P, P, C.c_double, C.c_int64,
                                   C.c_uint64, C.c_int64, P, P, C.c_int]
        L.om_integrate.restype = C.c_int
        L.om_trace.argtypes = [P, P, P, P, C.c_int, P, P]
        L.om_trace.restype = C.c_int
        L.om_geodesic_paths.argtypes = [P, C.c_int64, P, P, C.c_double, C.c_int64, P, P, C.c_int, P, P, P, P,
                                        P]
        L.om_geodesic_paths.restype = C.c_int
        L.om_fire.argtypes = [P, C.c_int64, P, P, P, P, P, P, C.c_double, C.c_int64, P, P, C.c_int]
        L.om_fire.restype = C.c_int
        L.om_philox4x32_10.argtypes = [P, P, P]
        L.om_normal_pair.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, P, P]
        _lib = L
    return _lib


class Stats(C.Structure):
    _fields_ = [("windows_created", C.c_int64), ("windows_propagated", C.c_int64),
                ("windows_dropped", C.c_int64), ("vertex_events", C.c_int64),
                ("sources", C.c_int64), ("queries", C.c_int64)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Potential(C.Structure):
    _fields_ = [("kind", C.c_int32), ("eps", C.c_double), ("sigma", C.c_double),
                ("r_cut", C.c_double), ("A", C.c_double)]


class Integrator(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dt", C.c_double), ("kT", C.c_double), ("lam", C.c_double),
                ("v0", C.c_double), ("Dr", C.c_double), ("mass", C.c_double),
                ("max_disp", C.c_double)]


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def potential(d: dict) -> Potential:
    return Potential(int(d["kind"]), float(d["eps"]), float(d["sigma"]), float(d["r_cut"]),
                     float(d.get("A", 1.0)))


def integrator(d: dict) -> Integrator:
    return Integrator(int(d["kind"]), float(d["dt"]), float(d["kT"]), float(d["lam"]),
                      float(d["v0"]), float(d["Dr"]), float(d["mass"]), float(d["max_disp"]))


class OracleMesh:
    def __init__(self, mesh):
        L = lib()
        self.mesh = mesh
        self._X = _f64(mesh.verts)
        self._F = _i32(mesh.faces)
        per = None if mesh.period is None else _f64(mesh.period)
        h = C.c_void_p()
        rc = L.om_mesh_create(_p(self._X), self._X.shape[0], _p(self._F), self._F.shape[0],
                              _p(per), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle mesh rejected (code {rc})")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.om_mesh_destroy(self.h)
            self.h = None

    @property
    def num_edges(self) -> int:
        return lib().om_mesh_num_edges(self.h)

    def vertex_info(self):
        nv = self.mesh.nv
        th = np.zeros(nv)
        ps = np.zeros(nv, np.uint8)
        bd = np.zeros(nv, np.uint8)
        lib().om_mesh_vertex_info(self.h, _p(th), _p(ps), _p(bd))
        return th, ps.astype(bool), bd.astype(bool)

    def face_frame(self, f: int) -> np.ndarray:
        out = np.zeros(9)
        lib().om_face_frame(self.h, int(f), _p(out))
        return out.reshape(3, 3)

    def world(self, face, bary) -> np.ndarray:
        face = _i32(np.atleast_1d(face))
        bary = _f64(np.atleast_2d(bary))
        out = np.zeros((face.shape[0], 3))
        for i in range(face.shape[0]):
            o = np.zeros(3)
            lib().om_world_position(self.h, int(face[i]), _p(np.ascontiguousarray(bary[i])), _p(o))
            out[i] = o
        return out

    def query(self, f0: int, b0, r_c: float, tf, tb, stats: bool = False):
        tf = _i32(np.atleast_1d(tf))
        tb = _f64(np.atleast_2d(tb))
        b0 = _f64(b0)
        d = np.zeros(tf.shape[0])
        t = np.zeros((tf.shape[0], 3))
        st = Stats()
        rc = lib().om_geodesic_query(self.h, int(f0), _p(b0), float(r_c), tf.shape[0], _p(tf),
                                     _p(tb), _p(d), _p(t), C.byref(st))
        if rc != 0:
            raise ValueError(f"oracle query failed ({rc})")
        return (d, t, st.asdict()) if stats else (d, t)

    def neighbors(self, face, bary, r_c: float, nthreads: int = 0, sources=None,
                  stats: bool = False):
        """CSR (row_start, j, dist, tangent world) of pairs with l_ij < r_c."""
        face = _i32(face)
        bary = _f64(bary)
        n = face.shape[0]
        st = Stats()
        np_ = C.c_int64(0)
        if sources is None:
            src = np.arange(n, dtype=np.int64)
        else:
            src = np.ascontiguousarray(sources, dtype=np.int64)
        ns = src.shape[0]
        cap = max(16, ns * 8)
        while True:
            rs = np.zeros(ns + 1, np.int64)
            j = np.zeros(cap, np.int32)
            d = np.zeros(cap)
            t = np.zeros((cap, 3))
            rc = lib().om_neighbors_subset(self.h, n, _p(face), _p(bary), float(r_c), ns, _p(src),
                                           cap, C.byref(np_), _p(rs), _p(j), _p(d), _p(t),
                                           int(nthreads), C.byref(st))
            if rc == -5:
                cap = int(np_.value)
                st = Stats()
                continue
            if rc != 0:
                raise ValueError(f"oracle neighbors failed ({rc})")
            k = int(np_.value)
            out = (rs, j[:k].copy(), d[:k].copy(), t[:k].copy())
            return (out + (st.asdict(),)) if stats else out

    def neighbors_gap(self, face, bary, r_c: float, nthreads: int = 0, sources=None):
        """(row_start, j, dist, tangent, gap): gap = extra length of the best rival path whose
        initial tangent differs (+inf when the geodesic is unique among the candidates).
        With `sources`, only those rows, in the order given."""
        face = _i32(face)
        bary = _f64(bary)
        n = face.shape[0]
        src = np.arange(n, dtype=np.int64) if sources is None else np.ascontiguousarray(sources, dtype=np.int64)
        ns = src.shape[0]
        np_ = C.c_int64(0)
        cap = max(16, ns * 8)
        while True:
            rs = np.zeros(ns + 1, np.int64)
            j = np.zeros(cap, np.int32)
            d = np.zeros(cap)
            t = np.zeros((cap, 3))
            g = np.zeros(cap)
            rc = lib().om_neighbors_gap(self.h, n, _p(face), _p(bary), float(r_c), ns, _p(src), cap,
                                        C.byref(np_), _p(rs), _p(j), _p(d), _p(t), _p(g), int(nthreads), None)
            if rc == -5:
                cap = int(np_.value)
                continue
            if rc != 0:
                raise ValueError(f"oracle neighbors failed ({rc})")
            k = int(np_.value)
            return rs, j[:k].copy(), d[:k].copy(), t[:k].copy(), g[:k].copy()

    def forces(self, face, bary, r_c: float, pot: dict, nthreads: int = 0):
        face = _i32(face)
        bary = _f64(bary)
        F = np.zeros((face.shape[0], 3))
        e = C.c_double(0.0)
        P = potential(pot)
        rc = lib().om_forces(self.h, face.shape[0], _p(face), _p(bary), float(r_c), C.byref(P),
                             _p(F), C.byref(e), int(nthreads))
        if rc != 0:
            raise ValueError(f"oracle forces failed ({rc})")
        return F, e.value

    def forces_subset(self, face, bary, r_c: float, pot: dict, sources, nthreads: int = 0):
        """Forces (len(sources) x 3) and half pair energies on the listed particles only."""
        face = _i32(face)
        bary = _f64(bary)
        src = np.ascontiguousarray(sources, dtype=np.int64)
        F = np.zeros((src.shape[0], 3))
        e = np.zeros(src.shape[0])
        P = potential(pot)
        rc = lib().om_forces_subset(self.h, face.shape[0], _p(face), _p(bary), float(r_c), C.byref(P),
                                    src.shape[0], _p(src), _p(F), _p(e), int(nthreads))
        if rc != 0:
            raise ValueError(f"oracle forces failed ({rc})")
        return F, e

    def shift(self, face: int, bary, disp3, carry=None):
        f = np.array([face], np.int32)
        b = _f64(bary).copy()
        d = _f64(disp3)
        nc = 0 if carry is None else np.atleast_2d(carry).shape[0]
        cr = None if carry is None else _f64(np.atleast_2d(carry)).copy()
        rc = lib().om_shift(self.h, _p(f), _p(b), _p(d), nc, _p(cr))
        if rc < 0:
            raise ValueError(f"oracle shift failed ({rc})")
        return int(f[0]), b, cr, rc

    def integrate(self, face, bary, vel, orient, force, pot: dict, integ: dict, r_c: float,
                  nsteps: int, seed: int = 0, step0: int = 0, noise=None, nthreads: int = 0):
        face = _i32(face).copy()
        bary = _f64(bary).copy()
        n = face.shape[0]
        vel = np.zeros((n, 3)) if vel is None else _f64(vel).copy()
        orient = np.zeros((n, 3)) if orient is None else _f64(orient).copy()
        force = np.zeros((n, 3)) if force is None else _f64(force).copy()
        P, I = potential(pot), integrator(integ)
        e = C.c_double(0.0)
        nz = None if noise is None else _f64(noise)
        rc = lib().om_integrate(self.h, n, _p(face), _p(bary), _p(vel), _p(orient), _p(force),
                                C.byref(P), C.byref(I), float(r_c), int(nsteps), int(seed),
                                int(step0), _p(nz), C.byref(e), int(nthreads))
        if rc != 0:
            raise ValueError(f"oracle integrate failed ({rc})")
        return dict(face=face, bary=bary, vel=vel, orient=orient, force=force, epot=e.value)


    def trace(self, face: int, bary, disp3, cap: int = 4096):
        """Polyline (world points: start, crossings, end) of the straightest walk from
        (face, bary) along disp3, and its end point (face, bary)."""
        f = C.c_int32(int(face))
        b = _f64(bary).copy()
        d = _f64(disp3)
        pts = np.zeros((cap, 3))
        n = C.c_int(0)
        rc = lib().om_trace(self.h, C.byref(f), _p(b), _p(d), int(cap), _p(pts), C.byref(n))
        if rc != 0:
            raise ValueError(f"oracle trace failed ({rc})")
        return pts[:min(n.value, cap)].copy(), n.value, f.value, b

    def geodesic_paths(self, face, bary, r_c: float, src, dst, cap: int = 512):
        """Shortest-path polylines of the pairs src[p] -> dst[p] (source first).  Returns
        (list of (npts, 3) arrays, empty when l >= r_c; legs; l; largest leg landing gap)."""
        face = _i32(face)
        bary = _f64(bary)
        src, dst = _i32(src), _i32(dst)
        np_ = src.shape[0]
        pts = np.zeros((np_, cap, 3))
        npts = np.zeros(np_, np.int32)
        legs = np.zeros(np_, np.int32)
        dist = np.zeros(np_)
        gap = np.zeros(np_)
        rc = lib().om_geodesic_paths(self.h, face.shape[0], _p(face), _p(bary), float(r_c), np_, _p(src), _p(dst),
                                     int(cap), _p(pts), _p(npts), _p(legs), _p(dist), _p(gap))
        if rc != 0:
            raise ValueError(f"oracle path extraction failed ({rc})")
        if np.any(npts > cap):
            raise ValueError("polyline longer than cap points")
        return [pts[p, :npts[p]].copy() for p in range(np_)], legs, dist, gap

    def fire(self, face, bary, vel, force, pot: dict, integ: dict, r_c: float, nsteps: int, state=None,
             nthreads: int = 0):
        """FIRE minimisation steps; force must hold the forces at the given positions.
        state = [dt, alpha, steps with P > 0] (default: the integrator's dt, 0.1, 0)."""
        face = _i32(face).copy()
        bary = _f64(bary).copy()
        n = face.shape[0]
        vel = np.zeros((n, 3)) if vel is None else _f64(vel).copy()
        force = _f64(force).copy()
        st = np.array([integ["dt"], 0.1, 0.0] if state is None else state, dtype=np.float64)
        P, I = potential(pot), integrator(integ)
        e = C.c_double(0.0)
        rc = lib().om_fire(self.h, n, _p(face), _p(bary), _p(vel), _p(force), C.byref(P), C.byref(I),
                           float(r_c), int(nsteps), _p(st), C.byref(e), int(nthreads))
        if rc != 0:
            raise ValueError(f"oracle fire failed ({rc})")
        return dict(face=face, bary=bary, vel=vel, force=force, state=st, epot=e.value)


def pair_energy(pot: dict, l: float) -> float:
    P = potential(pot)
    return lib().om_pair_energy(C.byref(P), float(l))


def pair_dudl(pot: dict, l: float) -> float:
    P = potential(pot)
    return lib().om_pair_dudl(C.byref(P), float(l))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().om_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def normal_pair(seed: int, particle: int, step: int):
    z0, z1 = C.c_double(), C.c_double()
    lib().om_normal_pair(seed, particle, step, C.byref(z0), C.byref(z1))
    return z0.value, z1.value


INF = math.inf
