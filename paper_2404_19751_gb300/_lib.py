"""ctypes binding of the C ABI in include/css.h (argument marshalling only).

Every computation runs in the CUDA library ``_build/libcss.so``; if it has not
been built (``python -c "import __graft_entry__ as g; g.build()"``) importing a
function from here raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcss.so")

OK = 0
ERR_NAMES = {-1: "INVALID_ARG", -2: "NONMANIFOLD", -3: "OOM", -4: "CUDA", -5: "CAPACITY",
             -6: "QUEUE_OVERFLOW", -7: "ITER_LIMIT", -8: "NO_DEVICE"}
FP64, FP32 = 0, 1
POT_HARMONIC, POT_WCA, POT_GAUSSIAN = 0, 1, 2
INT_NVE, INT_BD, INT_ABP, INT_GD, INT_FIRE = 0, 1, 2, 3, 4

SYMBOLS = ("css_create", "css_destroy", "css_last_error", "css_last_counters", "css_set_launch",
           "css_mesh_upload", "css_mesh_free", "css_mesh_counts", "css_particles_set",
           "css_particles_get", "css_particles_free", "css_geodesic_neighbors", "css_compute_forces",
           "css_integrate_step", "css_batch_create", "css_batch_step", "css_batch_free",
           "css_last_kernel_ms", "css_fma_peak", "css_particles_update", "css_get_launch", "css_autotune",
           "css_trace_geodesics", "css_geodesic_paths", "css_particles_set_step", "css_vhm_neighbors")


class CssError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Potential(C.Structure):
    _fields_ = [("kind", C.c_int32), ("eps", C.c_double), ("sigma", C.c_double),
                ("r_cut", C.c_double), ("A", C.c_double)]


class Launch(C.Structure):
    """Launch shape of the neighbour/force evaluation (see css_launch in css.h)."""
    _fields_ = [("warps_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32), ("tile", C.c_int32),
                ("shared_scale", C.c_int32), ("window_capacity", C.c_int32), ("window_capacity2", C.c_int32),
                ("warps2_per_sm", C.c_int32), ("occupancy", C.c_int32), ("table_capacity", C.c_int32),
                ("team", C.c_int32)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Integrator(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dt", C.c_double), ("kT", C.c_double), ("lam", C.c_double),
                ("v0", C.c_double), ("Dr", C.c_double), ("mass", C.c_double),
                ("max_disp", C.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library (raises when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing")
    L = C.CDLL(path)
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    sig = {
        "css_create": [C.POINTER(C.c_void_p), C.c_int, P],
        "css_destroy": [P],
        "css_last_error": [P],
        "css_last_counters": [P, P],
        "css_set_launch": [P, P],
        "css_get_launch": [P, P],
        "css_autotune": [P, P, I32, P, D, C.c_int, I32, I64, P, C.POINTER(D)],
        "css_trace_geodesics": [P, I64, P, P, P, I32, P, P, P, P],
        "css_geodesic_paths": [P, D, I64, P, P, I32, P, P, P, P, P],
        "css_particles_set_step": [P, I64],
        "css_mesh_upload": [P, P, I64, P, I64, P, C.POINTER(C.c_void_p)],
        "css_mesh_free": [P],
        "css_mesh_counts": [P, P],
        "css_particles_set": [P, P, I64, P, P, P, P, C.c_uint64, C.POINTER(C.c_void_p)],
        "css_particles_get": [P, P, P, P, P, P, P],
        "css_particles_free": [P],
        "css_geodesic_neighbors": [P, D, C.c_int, I64, C.POINTER(I64), P, P, P, P],
        "css_vhm_neighbors": [P, D, D, I64, C.POINTER(I64), P, P, P, P],
        "css_compute_forces": [P, P, D, C.c_int, P, P],
        "css_integrate_step": [P, P, P, D, C.c_int, I64, P, P],
        "css_batch_create": [P, P, I32, C.POINTER(C.c_void_p)],
        "css_batch_step": [P, P, P, D, C.c_int, I64],
        "css_batch_free": [P],
        "css_last_kernel_ms": [P, C.POINTER(D)],
        "css_fma_peak": [P, C.c_int, C.POINTER(D)],
        "css_particles_update": [P, P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.css_last_error.restype = C.c_char_p
    _lib = L
    return L


def _ptr(a) -> Optional[int]:
    """Raw pointer of a numpy array or a torch tensor (host or CUDA), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def _f64(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.int32)


class Context:
    def __init__(self, device: int = 0, stream: Optional[int] = None):
        L = load()
        h = C.c_void_p()
        self._check(L.css_create(C.byref(h), device, stream), None)
        self.h = h

    def _check(self, rc: int, h=True):
        if rc != OK:
            msg = ""
            if h is not None and getattr(self, "h", None):
                msg = load().css_last_error(self.h).decode()
            raise CssError(rc, msg)

    def check(self, rc: int):
        self._check(rc)

    def close(self):
        if getattr(self, "h", None):
            load().css_destroy(self.h)
            self.h = None

    def last_counters(self):
        out = np.zeros(6, np.int64)
        self.check(load().css_last_counters(self.h, out.ctypes.data))
        return dict(zip(["sources", "windows", "propagated", "pairs", "deferred", "retries"], out.tolist()))

    def last_kernel_ms(self) -> float:
        ms = C.c_double(0.0)
        self.check(load().css_last_kernel_ms(self.h, C.byref(ms)))
        return ms.value

    def fma_peak(self, precision: int) -> float:
        f = C.c_double(0.0)
        self.check(load().css_fma_peak(self.h, int(precision), C.byref(f)))
        return f.value

    def get_launch(self) -> dict:
        L = Launch()
        self.check(load().css_get_launch(self.h, C.byref(L)))
        return L.asdict()

    def set_launch(self, **kw):
        """Change fields of the launch shape (the others keep their values)."""
        cur = self.get_launch()
        unknown = set(kw) - set(cur)
        if unknown:
            raise KeyError(unknown)
        cur.update(kw)
        L = Launch(**{k: int(v) for k, v in cur.items()})
        self.check(load().css_set_launch(self.h, C.byref(L)))

    def autotune(self, sets, pot, r_c: float, precision: int, reps: int = 1, sample: int = 0):
        """Pick the fastest launch shape for these particle sets; returns (shape, ms)."""
        arr = (C.c_void_p * len(sets))(*[p.h.value for p in sets])
        P = _pot(pot)
        L = Launch()
        ms = C.c_double(0.0)
        self.check(load().css_autotune(self.h, arr, len(sets), C.byref(P), float(r_c), int(precision), int(reps),
                                       int(sample), C.byref(L), C.byref(ms)))
        return L.asdict(), ms.value


def create(device: int = 0, stream: Optional[int] = None) -> Context:
    return Context(device, stream)


class Mesh:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    def counts(self):
        out = np.zeros(4, np.int64)
        self.ctx.check(load().css_mesh_counts(self.h, out.ctypes.data))
        return dict(zip(["nv", "nf", "ne", "npseudo"], out.tolist()))

    def free(self):
        if self.h:
            load().css_mesh_free(self.h)
            self.h = None


def mesh_upload(ctx: Context, verts, faces, period: Optional[Sequence[float]] = None) -> Mesh:
    v, f = _f64(verts), _i32(faces)
    nv = v.shape[0]
    nf = f.shape[0]
    per = None if period is None else np.ascontiguousarray(period, np.float64)
    h = C.c_void_p()
    ctx.check(load().css_mesh_upload(ctx.h, _ptr(v), nv, _ptr(f), nf, _ptr(per), C.byref(h)))
    return Mesh(ctx, h)


class Particles:
    def __init__(self, ctx: Context, mesh: Mesh, h, n: int):
        self.ctx, self.mesh, self.h, self.n = ctx, mesh, h, n

    def free(self):
        if self.h:
            load().css_particles_free(self.h)
            self.h = None


def particles_set(ctx: Context, mesh: Mesh, face, bary, vel=None, orient=None, seed: int = 0) -> Particles:
    f, b, v, o = _i32(face), _f64(bary), _f64(vel), _f64(orient)
    n = f.shape[0]
    h = C.c_void_p()
    ctx.check(load().css_particles_set(ctx.h, mesh.h, n, _ptr(f), _ptr(b), _ptr(v), _ptr(o),
                                       int(seed), C.byref(h)))
    return Particles(ctx, mesh, h, n)


def particles_get(parts: Particles):
    n = parts.n
    out = dict(face=np.zeros(n, np.int32), bary=np.zeros((n, 3)), vel=np.zeros((n, 3)),
               orient=np.zeros((n, 3)), force=np.zeros((n, 3)))
    step = C.c_int64(0)
    parts.ctx.check(load().css_particles_get(parts.h, out["face"].ctypes.data, out["bary"].ctypes.data,
                                             out["vel"].ctypes.data, out["orient"].ctypes.data,
                                             out["force"].ctypes.data, C.byref(step)))
    out["step"] = step.value
    return out


def particles_update(parts: Particles, face=None, bary=None, vel=None, orient=None):
    f, b, v, o = _i32(face), _f64(bary), _f64(vel), _f64(orient)
    parts.ctx.check(load().css_particles_update(parts.h, _ptr(f), _ptr(b), _ptr(v), _ptr(o)))


def particles_set_step(parts: Particles, step: int):
    """Set the step counter (noise stream position), e.g. when resuming from a checkpoint."""
    parts.ctx.check(load().css_particles_set_step(parts.h, int(step)))


def particles_get_into(parts: Particles, face=None, bary=None, vel=None, orient=None, force=None):
    """Copy state into caller buffers (numpy or torch, host or device); None skips a field."""
    step = C.c_int64(0)
    parts.ctx.check(load().css_particles_get(parts.h, _ptr(face), _ptr(bary), _ptr(vel), _ptr(orient),
                                             _ptr(force), C.byref(step)))
    return step.value


def geodesic_neighbors(parts: Particles, r_c: float, precision: int = FP64, capacity: Optional[int] = None):
    """CSR (row_start, j, dist, tangent) of all ordered pairs with l_ij < r_c (host arrays)."""
    n = parts.n
    L = load()
    npairs = C.c_int64(0)
    cap = capacity if capacity is not None else (max(64, 32 * n) if math.isfinite(r_c) else max(1, n * (n - 1)))
    while True:
        rs = np.zeros(n + 1, np.int64)
        j = np.zeros(max(cap, 1), np.int32)
        d = np.zeros(max(cap, 1))
        t = np.zeros((max(cap, 1), 3))
        rc = L.css_geodesic_neighbors(parts.h, float(r_c), int(precision), int(cap), C.byref(npairs),
                                      rs.ctypes.data, j.ctypes.data, d.ctypes.data, t.ctypes.data)
        if rc == -5 and capacity is None:
            cap = int(npairs.value)
            continue
        parts.ctx.check(rc)
        k = int(npairs.value)
        return rs, j[:k], d[:k], t[:k]


def vhm_neighbors(parts: Particles, r_c: float, t_factor: float = 1.0, capacity: Optional[int] = None):
    """Approximate neighbours (heat-method distances, vector-heat tangents; see
    css_vhm_neighbors): CSR (row_start, j, dist, tangent) as host arrays."""
    n = parts.n
    L = load()
    npairs = C.c_int64(0)
    cap = capacity if capacity is not None else (max(64, 32 * n) if math.isfinite(r_c) else max(1, n * (n - 1)))
    while True:
        rs = np.zeros(n + 1, np.int64)
        j = np.zeros(max(cap, 1), np.int32)
        d = np.zeros(max(cap, 1))
        t = np.zeros((max(cap, 1), 3))
        rc = L.css_vhm_neighbors(parts.h, float(r_c), float(t_factor), int(cap), C.byref(npairs),
                                 rs.ctypes.data, j.ctypes.data, d.ctypes.data, t.ctypes.data)
        if rc == -5 and capacity is None:
            cap = int(npairs.value)
            continue
        parts.ctx.check(rc)
        k = int(npairs.value)
        return rs, j[:k], d[:k], t[:k]


def trace_geodesics(parts: Particles, src, tangent, length, max_points: int = 256):
    """Polylines of straightest geodesics (see css_trace_geodesics): returns a list of
    (points (k x 3), complete) and the end points (face, bary)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    tan = np.ascontiguousarray(tangent, dtype=np.float64).reshape(-1, 3)
    ln = np.ascontiguousarray(length, dtype=np.float64)
    n = src.shape[0]
    pts = np.zeros((max(n, 1), max_points, 3))
    npts = np.zeros(max(n, 1), np.int32)
    ef = np.zeros(max(n, 1), np.int32)
    eb = np.zeros((max(n, 1), 3))
    parts.ctx.check(load().css_trace_geodesics(parts.h, n, src.ctypes.data, tan.ctypes.data, ln.ctypes.data,
                                               int(max_points), pts.ctypes.data, npts.ctypes.data,
                                               ef.ctypes.data, eb.ctypes.data))
    paths = [(pts[k, :min(npts[k], max_points)].copy(), bool(npts[k] <= max_points)) for k in range(n)]
    return paths, ef[:n], eb[:n]


def geodesic_paths(parts: Particles, r_c: float, src, dst, max_points: int = 512):
    """Shortest-path polylines of the pairs src[k] -> dst[k], bends included (see
    css_geodesic_paths): returns (list of (k x 3) point arrays, source first, empty when
    l >= r_c; legs; distances; largest leg landing gap)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    n = src.shape[0]
    pts = np.zeros((max(n, 1), max_points, 3))
    npts = np.zeros(max(n, 1), np.int32)
    legs = np.zeros(max(n, 1), np.int32)
    dist = np.zeros(max(n, 1))
    gap = np.zeros(max(n, 1))
    parts.ctx.check(load().css_geodesic_paths(parts.h, float(r_c), n, src.ctypes.data, dst.ctypes.data,
                                              int(max_points), pts.ctypes.data, npts.ctypes.data, legs.ctypes.data,
                                              dist.ctypes.data, gap.ctypes.data))
    if np.any(npts[:n] > max_points):
        raise ValueError("a polyline has more than max_points points")
    return [pts[k, :npts[k]].copy() for k in range(n)], legs[:n], dist[:n], gap[:n]


def _pot(p) -> Potential:
    if isinstance(p, Potential):
        return p
    return Potential(int(p["kind"]), float(p["eps"]), float(p["sigma"]), float(p["r_cut"]), float(p.get("A", 1.0)))


def _integ(it) -> Integrator:
    if isinstance(it, Integrator):
        return it
    return Integrator(int(it["kind"]), float(it["dt"]), float(it["kT"]), float(it["lam"]), float(it["v0"]),
                      float(it["Dr"]), float(it["mass"]), float(it["max_disp"]))


def compute_forces(parts: Particles, pot, r_c: float, precision: int = FP64, out=None):
    """Forces (n x 3) and potential energy; out may be a host array or a CUDA tensor."""
    P = _pot(pot)
    F = np.zeros((parts.n, 3)) if out is None else out
    e = C.c_double(0.0)
    parts.ctx.check(load().css_compute_forces(parts.h, C.byref(P), float(r_c), int(precision), _ptr(F),
                                              C.byref(e)))
    return F, e.value


def integrate_step(parts: Particles, pot, integ, r_c: float, precision: int = FP64, n_steps: int = 1,
                   noise=None) -> float:
    P, I = _pot(pot), _integ(integ)
    nz = _f64(noise)
    e = C.c_double(0.0)
    parts.ctx.check(load().css_integrate_step(parts.h, C.byref(P), C.byref(I), float(r_c), int(precision),
                                              int(n_steps), _ptr(nz), C.byref(e)))
    return e.value


class Batch:
    def __init__(self, ctx: Context, h, sets):
        self.ctx, self.h, self.sets = ctx, h, sets

    def free(self):
        if self.h:
            load().css_batch_free(self.h)
            self.h = None


def batch_create(ctx: Context, sets: Sequence[Particles]) -> Batch:
    arr = (C.c_void_p * len(sets))(*[s.h.value for s in sets])
    h = C.c_void_p()
    ctx.check(load().css_batch_create(ctx.h, arr, len(sets), C.byref(h)))
    return Batch(ctx, h, list(sets))


def batch_step(batch: Batch, pot, integ, r_c: float, precision: int = FP32, n_steps: int = 1):
    P, I = _pot(pot), _integ(integ)
    batch.ctx.check(load().css_batch_step(batch.h, C.byref(P), C.byref(I), float(r_c), int(precision),
                                          int(n_steps)))


INF = math.inf
