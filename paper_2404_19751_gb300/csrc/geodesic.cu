// geodesic.cu -- cutoff geodesic neighbours and forces, one warp per source particle.
//
// Method (Sec. 2.2 and Sec. 3.1 of the paper): exact polyhedral geodesics from a
// source point by continuous window propagation.  A window is an interval of an
// edge together with a pseudo-source s (the source, or a boundary / flat / saddle
// vertex where shortest paths may bend) unfolded into the plane of that edge and
// the geodesic length sigma from the source to s; it carries the distance
// sigma + |x - s| to the points x it sees.  Each window is unfolded into the next
// face, its cone is cut by the two far edges into at most two child windows, each
// child is intersected with the windows already on its edge so every point keeps
// the smaller distance, vertices reached receive distance candidates, and
// pseudo-source vertices start windows on their opposite edges.  Windows whose
// smallest distance is >= r_c are dropped (the Euclidean-lower-bound submesh of
// Sec. 3.1 becomes this cutoff stop).  Afterwards every particle in a reached face
// is evaluated: minimum over the direct segment, the windows entering its face
// whose cone contains it, and paths through the face's vertices; the force
// F_i = sum_j U'(l_ij) t_ij is accumulated in the same pass.
//
// GPU organisation: one warp owns one source at a time (persistent grid pulling
// sources, in Morton order of their faces, from a device counter).  Each wave takes
// up to 32 pending windows among those with the smallest keys (a relaxed priority
// order; exact because every window only ever carries the length of a real path and
// trimming keeps the pointwise minimum), unfolds them in parallel, then inserts the
// children: lanes that target the same edge are grouped with __match_any_sync and take
// turns, lanes on different edges trim in parallel.  A pseudo-source vertex emits its
// windows once no pending key is below its distance.  Two passes: the first keeps the
// per-warp hash tables (edge list heads, pseudo-source vertices, face set) in shared
// memory; a source whose patch overflows them or the window pool is deferred to a second
// pass with generation-tagged tables in the warp's global-memory workspace slice.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "css_internal.h"

namespace {

using css::DMesh;
using css::HeRec;

constexpr int WIN_ALIVE = 1;
constexpr int WIN_DONE = 2;    // already unfolded
constexpr int WIN_FIXED = 4;   // tangent fixed (descends from a pseudo-source vertex)
constexpr int MAXP = 4;        // interval pieces one insertion may hold
constexpr int MAX_WARPS_CTA = 16;

// Window record.  The pseudo-source s and its geodesic length sigma are the accumulated
// unfolded source state and stay FP64 in both forms; the FP32 form also keeps FP32 copies
// of them for its arithmetic, so that a window is 64 bytes and FP64 instructions are only
// issued for the unfolding transform of s and for near-degenerate decisions.
struct Win32 {
    double sx, sy, sig;
    float fsx, fsy, fsig;
    float b0, b1;      // interval along the half-edge
    float ta, tb;      // image of the source-face x axis (direct) or fixed tangent
    int32_t he, next, flags;
};
struct Win64 {
    double sx, sy, sig;
    double b0, b1, ta, tb;
    int32_t he, next, flags;
    int32_t pv;        // pseudo-source vertex (-1: the source); set by the path kernel only
};
template <class R>
struct WinT;
template <>
struct WinT<float> {
    using type = Win32;
};
template <>
struct WinT<double> {
    using type = Win64;
};
template <class R>
using Win = typename WinT<R>::type;

__device__ __forceinline__ float fsx(const Win32& w) { return w.fsx; }
__device__ __forceinline__ float fsy(const Win32& w) { return w.fsy; }
__device__ __forceinline__ float fsig(const Win32& w) { return w.fsig; }
__device__ __forceinline__ double fsx(const Win64& w) { return w.sx; }
__device__ __forceinline__ double fsy(const Win64& w) { return w.sy; }
__device__ __forceinline__ double fsig(const Win64& w) { return w.sig; }
__device__ __forceinline__ void set_fast(Win32& w) { w.fsx = (float)w.sx; w.fsy = (float)w.sy; w.fsig = (float)w.sig; }
__device__ __forceinline__ void set_fast(Win64&) {}

template <class R>
struct Tol;
template <>
struct Tol<double> {
    static constexpr double w = 1e-12;   // relative interval width / endpoint tolerance
};
template <>
struct Tol<float> {
    static constexpr float w = 2e-6f;
};

// relative distance difference below which two windows tie
template <class R>
struct Tie;
template <>
struct Tie<double> {
    static constexpr double rel = 1e-13;
};
template <>
struct Tie<float> {
    static constexpr double rel = 1e-6;
};

struct WarpSm {
    int nwin, npend, nface, nemit, err;
    unsigned emin;    // a lower bound on the distances of the queued emitting vertices (FP32 bits)
    int ncar;         // windows held over to the next wave's insertion rounds
    unsigned cmin;    // a lower bound on their keys (FP32 bits)
    int nstg;         // windows an emission round left in a caller's buffer
    int sel[32];      // window ids picked for the current wave
};

// Per-warp working state.  The keyed tables (edge heads, pseudo-source vertices, face set)
// live either in shared memory -- plain 32-bit keys, cleared for every source, for patches
// that fit -- or in the warp's global workspace slice with generation-tagged 64-bit keys;
// the window pool is always in the global slice.
// Per vertex of the table, how its distance was reached, for the path extraction: the
// previous node of its path (a pseudo-source vertex, -1 = the source), 4 * face + corner of
// a face holding the vertex whose layout the direction is written in, the unit direction
// from the vertex towards that node and the leg's length.  Present only in the path
// instantiation of the kernel.
template <bool L>
struct WsLinks {};
template <>
struct WsLinks<true> {
    int32_t* lpar;
    int32_t* lfk;
    double* ldir;
    double* llen;
};

template <class R, int SH>
struct Ws : WsLinks<SH == 2> {
    static constexpr bool shared = SH == 1;   // keyed tables in shared memory (else global, tagged)
    static constexpr bool links = SH == 2;    // also records how each vertex was reached (paths)
    int32_t* sekey;
    int32_t* svkey;
    int32_t* sfkey;
    unsigned long long* ekey;
    int32_t* ehead;
    unsigned long long* vkey;
    double* vdist;
    R* vtan;
    int32_t* vvid;
    int32_t* vflag;
    unsigned long long* fkey;
    int32_t* flist;
    Win<R>* win;
    int32_t* emit;
    int32_t* pq;      // pending (not yet unfolded) window ids
    float* pk;        // their keys when queued (lower bounds: trimming only raises a key)
    int log_eh, log_vh, log_fh, wcap, fcap, emcap;
    uint32_t gen;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

template <class R>
__host__ __device__ inline size_t ws_layout(int log_eh, int log_vh, int log_fh, int wcap, int fcap, int emcap,
                                            size_t* off) {
    size_t o = 0;
    const size_t EH = 1ull << log_eh, VH = 1ull << log_vh, FH = 1ull << log_fh;
    off[0] = o; o = al16(o + EH * 8);          // ekey
    off[1] = o; o = al16(o + EH * 4);          // ehead
    off[2] = o; o = al16(o + VH * 8);          // vkey
    off[3] = o; o = al16(o + VH * 8);          // vdist
    off[4] = o; o = al16(o + VH * 2 * sizeof(R));  // vtan
    off[5] = o; o = al16(o + VH * 4);          // vvid
    off[6] = o; o = al16(o + VH * 4);          // vflag
    off[7] = o; o = al16(o + FH * 8);          // fkey
    off[8] = o; o = al16(o + (size_t)fcap * 4);   // flist
    off[9] = o; o = al16(o + (size_t)wcap * sizeof(Win<R>));
    off[10] = o; o = al16(o + (size_t)emcap * 4);
    off[11] = o; o = al16(o + (size_t)wcap * 4);   // pq
    off[12] = o; o = al16(o + (size_t)wcap * 4);   // pk
    return o;
}

template <class R, int SH>
__device__ inline Ws<R, SH> ws_bind(const cssi::GeoWs& g, int warp) {
    size_t off[13];
    ws_layout<R>(g.log_eh, g.log_vh, g.log_fh, g.wcap, g.fcap, g.emcap, off);
    char* b = g.base + (size_t)warp * g.stride;
    Ws<R, SH> w;
    w.ekey = (unsigned long long*)(b + off[0]);
    w.ehead = (int32_t*)(b + off[1]);
    w.vkey = (unsigned long long*)(b + off[2]);
    w.vdist = (double*)(b + off[3]);
    w.vtan = (R*)(b + off[4]);
    w.vvid = (int32_t*)(b + off[5]);
    w.vflag = (int32_t*)(b + off[6]);
    w.fkey = (unsigned long long*)(b + off[7]);
    w.flist = (int32_t*)(b + off[8]);
    w.win = (Win<R>*)(b + off[9]);
    w.emit = (int32_t*)(b + off[10]);
    w.pq = (int32_t*)(b + off[11]);
    w.pk = (float*)(b + off[12]);
    w.log_eh = g.log_eh; w.log_vh = g.log_vh; w.log_fh = g.log_fh;
    w.wcap = g.wcap; w.fcap = g.fcap; w.emcap = g.emcap;
    w.gen = 0;
    w.sekey = w.svkey = w.sfkey = nullptr;
    if constexpr (SH == 2) {
        const size_t VH = (size_t)1 << g.log_vh;
        char* lb = g.lbase + (size_t)warp * g.lstride;
        w.lpar = (int32_t*)lb;
        w.lfk = (int32_t*)(lb + al16(VH * 4));
        w.ldir = (double*)(lb + 2 * al16(VH * 4));
        w.llen = w.ldir + 2 * VH;
    }
    return w;
}

// shared-memory tables of one warp.  Their sizes are the base sizes below times a
// power-of-two scale chosen per launch (larger patches, fewer warps per SM); a source
// whose patch overflows them is handed to the second, global-table pass.
constexpr int SH_LOG_EH = 9, SH_LOG_VH = 8, SH_LOG_FH = 9;
constexpr int SH_FCAP = 512, SH_EMCAP = 256;

__host__ __device__ inline int sh_log2(int scale) {
    int l = 0;
    while ((1 << l) < scale) ++l;
    return l;
}

template <class R>
__host__ __device__ inline size_t sh_bytes_per_warp(int scale) {
    const size_t s = (size_t)1 << sh_log2(scale);
    return s * ((size_t)(1 << SH_LOG_EH) * 8 + (size_t)(1 << SH_LOG_VH) * (4 + 8 + 2 * sizeof(R) + 4) +
                (size_t)(1 << SH_LOG_FH) * 4 + (size_t)SH_FCAP * 4 + (size_t)SH_EMCAP * 4);
}

template <class R, int SH>
__device__ inline void ws_bind_shared(Ws<R, SH>& w, unsigned char* base, int scale) {
    const int ls = sh_log2(scale);
    const int eh = 1 << (SH_LOG_EH + ls), vh = 1 << (SH_LOG_VH + ls), fh = 1 << (SH_LOG_FH + ls);
    unsigned char* p = base;
    w.sekey = (int32_t*)p; p += eh * 4;
    w.ehead = (int32_t*)p; p += eh * 4;
    w.vdist = (double*)p; p += vh * 8;
    w.vtan = (R*)p; p += vh * 2 * sizeof(R);
    w.svkey = (int32_t*)p; p += vh * 4;
    w.vflag = (int32_t*)p; p += vh * 4;
    w.sfkey = (int32_t*)p; p += fh * 4;
    w.flist = (int32_t*)p; p += (SH_FCAP << ls) * 4;
    w.emit = (int32_t*)p;
    w.vvid = w.svkey;   // the key is the vertex id
    w.log_eh = SH_LOG_EH + ls; w.log_vh = SH_LOG_VH + ls; w.log_fh = SH_LOG_FH + ls;
    w.fcap = SH_FCAP << ls; w.emcap = SH_EMCAP << ls;
}

__device__ __forceinline__ int sh_insert(int32_t* keys, int logcap, int32_t key, bool& claimed) {
    const uint32_t mask = (1u << logcap) - 1u;
    uint32_t slot = ((uint32_t)key * 2654435761u) >> (32 - logcap);
    claimed = false;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        int32_t cur = *(volatile int32_t*)(keys + slot);
        if (cur == key) return (int)slot;
        if (cur == -1) {
            const int32_t prev = atomicCAS(keys + slot, -1, key);
            if (prev == -1) { claimed = true; return (int)slot; }
            if (prev == key) return (int)slot;
        }
        slot = (slot + 1u) & mask;
    }
    return -1;
}

__device__ __forceinline__ int sh_find(const int32_t* keys, int logcap, int32_t key) {
    const uint32_t mask = (1u << logcap) - 1u;
    uint32_t slot = ((uint32_t)key * 2654435761u) >> (32 - logcap);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t cur = *(volatile const int32_t*)(keys + slot);
        if (cur == key) return (int)slot;
        if (cur == -1) return -1;
        slot = (slot + 1u) & mask;
    }
    return -1;
}

template <class R, int SH>
__device__ __forceinline__ int ws_eins(Ws<R, SH>& ws, int32_t key, bool& claimed) {
    return ws.shared ? sh_insert(ws.sekey, ws.log_eh, key, claimed) : css::ht_insert(ws.ekey, ws.log_eh, ws.gen, key, claimed);
}
template <class R, int SH>
__device__ __forceinline__ int ws_efind(const Ws<R, SH>& ws, int32_t key) {
    return ws.shared ? sh_find(ws.sekey, ws.log_eh, key) : css::ht_find(ws.ekey, ws.log_eh, ws.gen, key);
}
template <class R, int SH>
__device__ __forceinline__ int ws_vins(Ws<R, SH>& ws, int32_t key, bool& claimed) {
    return ws.shared ? sh_insert(ws.svkey, ws.log_vh, key, claimed) : css::ht_insert(ws.vkey, ws.log_vh, ws.gen, key, claimed);
}
template <class R, int SH>
__device__ __forceinline__ int ws_vfind(const Ws<R, SH>& ws, int32_t key) {
    return ws.shared ? sh_find(ws.svkey, ws.log_vh, key) : css::ht_find(ws.vkey, ws.log_vh, ws.gen, key);
}
template <class R, int SH>
__device__ __forceinline__ int ws_fins(Ws<R, SH>& ws, int32_t key, bool& claimed) {
    return ws.shared ? sh_insert(ws.sfkey, ws.log_fh, key, claimed) : css::ht_insert(ws.fkey, ws.log_fh, ws.gen, key, claimed);
}

// forget the previous source's shared tables
template <class R, int SH>
__device__ __forceinline__ void ws_clear_shared(Ws<R, SH>& ws, int lane) {
    if constexpr (SH == 1) {
        for (int k = lane; k < (1 << ws.log_eh); k += 32) ws.sekey[k] = -1;
        for (int k = lane; k < (1 << ws.log_vh); k += 32) ws.svkey[k] = -1;
        for (int k = lane; k < (1 << ws.log_fh); k += 32) ws.sfkey[k] = -1;
        __syncwarp();
    }
}

// ------------------------------------------------------------------ window geometry
// The "fast" type F is the form's arithmetic type: float in the FP32 form, double in FP64.

// half-edge geometry in the form's precision
template <class R>
struct HeF {
    R L, cx, cy, cl, sl, cr, sr;
};
template <class R>
__device__ __forceinline__ HeF<R> he_fast(const DMesh& m, int h, const HeRec& r);
template <>
__device__ __forceinline__ HeF<double> he_fast<double>(const DMesh&, int, const HeRec& r) {
    return HeF<double>{r.L, r.cx, r.cy, r.cl, r.sl, r.cr, r.sr};
}
template <>
__device__ __forceinline__ HeF<float> he_fast<float>(const DMesh& m, int h, const HeRec&) {
    const css::HeRec32 q = m.he32[h];
    return HeF<float>{q.L, q.cx, q.cy, q.cl, q.sl, q.cr, q.sr};
}

template <class R>
__device__ __forceinline__ void face_corner_f(const DMesh& m, int f, int k, R& x, R& y);
template <>
__device__ __forceinline__ void face_corner_f<double>(const DMesh& m, int f, int k, double& x, double& y) {
    css::face_corner(m, f, k, x, y);
}
template <>
__device__ __forceinline__ void face_corner_f<float>(const DMesh& m, int f, int k, float& x, float& y) {
    k = (k >= 3) ? k - 3 : k;
    if (k == 0) { x = 0.f; y = 0.f; }
    else if (k == 1) { x = m.lay32[3 * f]; y = 0.f; }
    else { x = m.lay32[3 * f + 1]; y = m.lay32[3 * f + 2]; }
}

// smallest distance the window carries over its interval
template <class R>
__device__ __forceinline__ R win_key(const Win<R>& w) {
    const R sx = fsx(w), sy = fsy(w);
    const R x = sx < w.b0 ? w.b0 : (sx > w.b1 ? w.b1 : sx);
    const R dx = x - sx;
    return fsig(w) + sqrt(dx * dx + sy * sy);
}

// distance carried to the point (px, py) of the window frame, form precision
template <class R>
__device__ __forceinline__ R win_dist(const Win<R>& w, R px, R py) {
    const R dx = px - fsx(w), dy = py - fsy(w);
    return fsig(w) + sqrt(dx * dx + dy * dy);
}

// the same in FP64 whatever the form: vertex distances become the sigma of later
// pseudo-sources and decide near-ties between path families
template <class R>
__device__ __forceinline__ double win_dist_exact(const Win<R>& w, double px, double py) {
    const double dx = px - w.sx, dy = py - w.sy;
    return w.sig + sqrt(dx * dx + dy * dy);
}

template <class R>
__device__ __forceinline__ void win_tangent(const Win<R>& w, R px, R py, R& tx, R& ty) {
    if (w.flags & WIN_FIXED) { tx = w.ta; ty = w.tb; return; }
    R dx = px - fsx(w), dy = py - fsy(w);
    const R n = sqrt(dx * dx + dy * dy);
    dx /= n; dy /= n;
    tx = dx * w.ta + dy * w.tb;
    ty = -dx * w.tb + dy * w.ta;
}

// a pseudo-source on the edge line sees the face beyond only through its own position
template <class R>
__device__ __forceinline__ bool win_degen(const Win<R>& w, R L) { return fsy(w) > (R)-1e-13 * L; }
template <class R>
__device__ __forceinline__ bool win_degen_sees(const Win<R>& w, R L) {
    const R tol = (R)1e-12 * L;
    return fsx(w) >= w.b0 - tol && fsx(w) <= w.b1 + tol;
}

// parameter in [0,1] along A->B hit by the ray from s through (X, 0)
template <class R>
__device__ __forceinline__ R ray_hit(R sx, R sy, R X, R ax, R ay, R bx, R by) {
    const R dx = X - sx, dy = -sy;
    const R ex = bx - ax, ey = by - ay;
    const R den = ex * dy - ey * dx;
    const R qx = sx - ax, qy = sy - ay;
    const R mu = den != (R)0 ? (qx * dy - qy * dx) / den : (R)0;
    return mu < (R)0 ? (R)0 : (mu > (R)1 ? (R)1 : mu);
}

// relative widening of child intervals computed with FP32 ray intersections, so that
// rounding never opens a gap between neighbouring windows (an overlap is resolved exactly by
// the trimming, a gap would hand its wedge to a longer path family)
template <class R>
struct Widen;
template <>
struct Widen<double> {
    static constexpr double mu = 0.0;
};
template <>
struct Widen<float> {
    static constexpr float mu = 8.0f * 1.1920929e-7f;
};

// how a candidate reaches its vertex (path kernel only): see WsLinks
template <bool L>
struct VLink {};
template <>
struct VLink<true> {
    int32_t par, fk;
    double dx, dy, len;
};

template <class R, bool L = false>
struct VCand : VLink<L> {
    int32_t v;
    int32_t fixed;   // tangent comes from a pseudo-source path
    double d;        // exact FP64 length
    R tx, ty;
    float back;      // direction of the path's last leg, seen from the vertex, as a cumulative
                     // corner angle (DMesh::cang); NaN where it is not known
};

// Cumulative angle at a vertex of the direction g, given the vertex's corner hc whose first
// edge runs along e (both in one face layout); NaN when g is too short to have a reliable
// direction or the corner has no cumulative angle.
__device__ __forceinline__ float back_angle(const DMesh& m, int hc, double ex, double ey, double gx, double gy,
                                            double scale) {
    if (hc < 0 || !(gx * gx + gy * gy > 1e-12 * scale * scale)) return __int_as_float(0x7fffffff);
    return m.cang[hc].x + atan2f((float)(ex * gy - ey * gx), (float)(ex * gx + ey * gy));
}

// The link of the point (X, Y) of window W's half-edge frame straight back to W's
// pseudo-source: which = 2 the far corner of the face W enters (the direction lies in that
// face); 0 / 1 the start / end vertex of W's edge (the direction points into the face on
// the other side of the edge and is written in that face); -1 a point inside the face W
// enters (corner slot 3).
__device__ void win_link(const DMesh& m, const Win64& W, double X, double Y, int which, VLink<true>& l) {
    const int h = W.he, f = h / 3, k = h - 3 * f;
    const double a = W.sx - X, b = W.sy - Y, n = sqrt(a * a + b * b);
    const double ua = n > 0.0 ? a / n : 1.0, ub = n > 0.0 ? b / n : 0.0;
    l.par = W.pv;
    l.len = n;
    int g = f, kg = k, kc = which == 2 ? (k == 0 ? 2 : k - 1) : 3;
    double va = ua, vb = ub;
    if ((which == 0 || which == 1) && m.twin[h] >= 0) {
        const int tw = m.twin[h];   // runs from W's end vertex to its start vertex
        g = tw / 3;
        kg = tw - 3 * g;
        kc = which == 0 ? (kg == 2 ? 0 : kg + 1) : kg;
        va = -ua;
        vb = -ub;
    }
    double ax, ay, bx, by;
    css::face_corner(m, g, kg, ax, ay);
    css::face_corner(m, g, kg + 1, bx, by);
    const double L = sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
    const double ex = (bx - ax) / L, ey = (by - ay) / L;
    l.dx = va * ex - vb * ey;
    l.dy = va * ey + vb * ex;
    l.fk = 4 * g + kc;
}

// Unfold window W into the next face: distance candidates for the pseudo-source vertices it
// reaches (paths through any other vertex can be shortened, Sec. 2.2) and at most two children.
template <class R, bool L>
__device__ __forceinline__ void propagate(const DMesh& m, const Win<R>& W, double rc, VCand<R, L>* vc, int& nvc,
                                       Win<R>* ch, int& nch) {
    nvc = 0;
    nch = 0;
    const int h = W.he;
    const int f = h / 3;
    const int k = h - 3 * f;
    const HeRec r = m.he[h];
    const HeF<R> q = he_fast<R>(m, h, r);
    const int k1 = (k == 2) ? 0 : k + 1, k2 = (k == 0) ? 2 : k - 1;
    const int32_t vu = m.fv[h], vv = m.fv[3 * f + k1], vcid = m.fv[3 * f + k2];
    const R tolv = (R)Tol<R>::w * q.L;
    const R sx = fsx(W), sy = fsy(W);
    const bool degen = win_degen<R>(W, q.L);
    const bool sees = !degen || win_degen_sees<R>(W, q.L);
    // occlusion predicate: where the ray s -> c crosses the edge line; in the FP32 form it is
    // re-evaluated in FP64 when it falls within 1e-5 L of an interval end
    R xc = (R)0;
    if (!degen) {
        xc = sx + (q.cx - sx) * (-sy) / (q.cy - sy);
        if (sizeof(R) == sizeof(float) && (fabs(xc - W.b0) < (R)1e-5 * q.L || fabs(xc - W.b1) < (R)1e-5 * q.L))
            xc = (R)(W.sx + (r.cx - W.sx) * (-W.sy) / (r.cy - W.sy));
    }
    // vertex candidates in the order start of the edge, end of the edge, far corner (one copy
    // of the candidate code)
    const bool take0 = W.b0 <= tolv && m.pseudo[vu];
    const bool take1 = W.b1 >= q.L - tolv && m.pseudo[vv];
    const bool take2 = sees && (degen || (xc >= W.b0 - tolv && xc <= W.b1 + tolv)) && m.pseudo[vcid];
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
        if (!(a == 0 ? take0 : (a == 1 ? take1 : take2))) continue;
        const double X = a == 0 ? 0.0 : (a == 1 ? r.L : r.cx), Y = a == 2 ? r.cy : 0.0;
        const R Xf = a == 0 ? (R)0 : (a == 1 ? q.L : q.cx), Yf = a == 2 ? q.cy : (R)0;
        VCand<R, L>& c = vc[nvc++];
        c.v = a == 0 ? vu : (a == 1 ? vv : vcid);
        c.fixed = W.flags & WIN_FIXED;
        c.d = win_dist_exact<R>(W, X, Y);
        win_tangent<R>(W, Xf, Yf, c.tx, c.ty);
        // the last leg back to the pseudo-source: at the start vertex it leaves below corner
        // h's first edge (u -> v), at the end vertex it lies in the corner of the face across
        // the edge (first edge v -> u), at the far corner inside corner c (first edge c -> u)
        c.back = degen ? __int_as_float(0x7fffffff)
                       : back_angle(m, a == 0 ? h : (a == 1 ? m.twin[h] : 3 * f + k2), a == 0 ? 1.0 : (a == 1 ? -1.0 : -r.cx),
                                    a == 2 ? -r.cy : 0.0, W.sx - X, W.sy - Y, r.L);
        if constexpr (L) win_link(m, W, X, Y, a, c);
    }
    if (!sees) return;
    // the children across the far edges: side 0 the edge u -> c (origin u, turned by
    // -angle(c)), side 1 the edge c -> v (origin c, turned by -angle(v - c)); one copy of the
    // child code
#pragma unroll 1
    for (int a = 0; a < 2; ++a) {
        const int tw = a == 0 ? r.tl : r.tr;
        if (tw < 0 || !(degen || (a == 0 ? xc > W.b0 : xc < W.b1))) continue;
        const R ax = a == 0 ? (R)0 : q.cx, ay = a == 0 ? (R)0 : q.cy;
        const R bx = a == 0 ? q.cx : q.L, by = a == 0 ? q.cy : (R)0;
        const R co = a == 0 ? q.cl : q.cr, si = a == 0 ? q.sl : q.sr;
        R mu0 = (R)0, mu1 = (R)1;
        if (!degen) {
            mu0 = (a == 1 && W.b0 <= xc) ? (R)0 : ray_hit<R>(sx, sy, W.b0, ax, ay, bx, by);
            mu1 = (a == 0 && W.b1 >= xc) ? (R)1 : ray_hit<R>(sx, sy, W.b1, ax, ay, bx, by);
            mu0 -= Widen<R>::mu; mu1 += Widen<R>::mu;
        }
        Win<R>& c = ch[nch];
        c = W;
        c.he = tw;
        const double dco = a == 0 ? r.cl : r.cr, dsi = a == 0 ? r.sl : r.sr;
        const double px = a == 0 ? W.sx : W.sx - r.cx, py = a == 0 ? W.sy : W.sy - r.cy;   // FP64
        c.sx = px * dco + py * dsi;
        c.sy = -px * dsi + py * dco;
        if (c.sy > 0.0) c.sy = 0.0;
        set_fast(c);
        if (!(W.flags & WIN_FIXED)) {
            c.ta = W.ta * co + W.tb * si;
            c.tb = -W.ta * si + W.tb * co;
        }
        const R Le = (bx - ax) * co + (by - ay) * si;   // length of the child's edge
        c.b0 = mu0 * Le; c.b1 = mu1 * Le;
        c.flags = (W.flags & WIN_FIXED) | WIN_ALIVE;
        if ((double)win_key<R>(c) < rc) ++nch;
    }
}


// Points x in (lo, hi) where two windows carry equal distance: |x-a| - |x-b| = sb - sa squared
// twice (FP64 in both forms: this is the near-degenerate intersection predicate).  Spurious
// roots only add breakpoints; the winner of each piece is decided by evaluation.
__device__ int equal_points(double ax, double ay, double sa, double bx, double by, double sb, double lo, double hi,
                            double& r0, double& r1) {
    const double del = sb - sa;
    const double al = bx - ax;
    const double be = (ax * ax + ay * ay) - (bx * bx + by * by) - del * del;
    const double c2 = del * del - al * al;
    const double c1 = -(2.0 * del * del * bx + al * be);
    const double c0 = del * del * (bx * bx + by * by) - 0.25 * be * be;
    double cand0 = 0.0, cand1 = 0.0;
    int nc = 0;
    const double scale = fabs(c2) + fabs(c1) / (fabs(hi) + fabs(lo) + 1e-300) + 1e-300;
    if (fabs(c2) <= 1e-14 * scale) {
        if (c1 != 0.0) { cand0 = -c0 / c1; nc = 1; }
    } else {
        double disc = c1 * c1 - 4.0 * c2 * c0;
        if (disc < 0.0) disc = 0.0;
        const double sq = sqrt(disc);
        const double qq = -0.5 * (c1 + (c1 >= 0.0 ? sq : -sq));
        if (qq != 0.0) { cand0 = qq / c2; cand1 = c0 / qq; nc = 2; }
        else { cand0 = -c1 / (2.0 * c2); nc = 1; }
    }
    int n = 0;
    const bool ok0 = nc > 0 && cand0 > lo && cand0 < hi;
    const bool ok1 = nc > 1 && cand1 > lo && cand1 < hi;
    if (ok0 && ok1) { r0 = fmin(cand0, cand1); r1 = fmax(cand0, cand1); n = 2; }
    else if (ok0) { r0 = cand0; n = 1; }
    else if (ok1) { r0 = cand1; n = 1; }
    return n;
}

// ---- register-resident interval lists (sorted, disjoint, at most MAXP)
// Every index is resolved by unrolled compare-and-select so the lists never spill to
// local memory.  When a list is full, `cover` decides: true extends the last interval over
// the gap (a window that keeps more than it must only costs work: every window carries real
// path lengths), false drops the new interval (used for the parts a window loses, so it
// never loses too much).
template <class R>
struct Ivl {
    R a[MAXP], b[MAXP];
    int n;
};

template <class R>
__device__ __forceinline__ R ivl_get(const R (&v)[MAXP], int i) {
    R r = v[0];
#pragma unroll
    for (int k = 1; k < MAXP; ++k)
        if (i == k) r = v[k];
    return r;
}
template <class R>
__device__ __forceinline__ void ivl_set(R (&v)[MAXP], int i, R x) {
#pragma unroll
    for (int k = 0; k < MAXP; ++k)
        if (i == k) v[k] = x;
}
template <class R>
__device__ __forceinline__ void ivl_add(Ivl<R>& L, R x0, R x1, bool cover = true) {
    if (!(x1 > x0)) return;
    if (L.n > 0) {
        const R lb = ivl_get<R>(L.b, L.n - 1);
        if (x0 <= lb) { if (x1 > lb) ivl_set<R>(L.b, L.n - 1, x1); return; }
    }
    if (L.n < MAXP) { ivl_set<R>(L.a, L.n, x0); ivl_set<R>(L.b, L.n, x1); ++L.n; }
    else if (cover) L.b[MAXP - 1] = x1;
}

// a[i] = x for a runtime index into a register array (predicated moves, no local memory)
template <class T, int N>
__device__ __forceinline__ void reg_set(T (&a)[N], int i, const T& x) {
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (k == i) a[k] = x;
}

template <class R, int SH>
__device__ __forceinline__ void face_add(Ws<R, SH>& ws, WarpSm& sm, int32_t f) {
    bool claimed;
    int s = ws_fins<R>(ws, f, claimed);
    if (s < 0) { atomicOr(&sm.err, css::ST_HASH_OVERFLOW); return; }
    if (claimed) {
        int p = atomicAdd(&sm.nface, 1);
        if (p < ws.fcap) ws.flist[p] = f;
        else atomicOr(&sm.err, css::ST_HASH_OVERFLOW);
    }
}

template <class R>
__device__ __forceinline__ int win_alloc(WarpSm& sm, int wcap) {
    int p = atomicAdd(&sm.nwin, 1);
    if (p >= wcap) { atomicOr(&sm.err, css::ST_WIN_OVERFLOW); return -1; }
    return p;
}

// queue a window that still has to be unfolded (each window is queued at most once, so
// the queue never holds more entries than the pool)
template <class R, int SH>
__device__ __forceinline__ void push_pending(Ws<R, SH>& ws, WarpSm& sm, int id, float key) {
    const int p = atomicAdd(&sm.npend, 1);
    ws.pq[p] = id;
    ws.pk[p] = key;
}

// Outcome of comparing two windows on an overlap [lo, hi]: one of them carries the
// smaller distance everywhere, or the exact FP64 split is needed.
enum { CMP_EXISTING = 0, CMP_CANDIDATE = 1, CMP_SPLIT = 2 };

// FP32 dominance test with rigorous margins: the distance difference D(x) is bounded from
// its endpoint values and from bounds on its derivative (each distance's derivative along the
// edge is monotone in x), with a rounding margin E on every evaluated difference.
__device__ __forceinline__ int dominance_f32(float csx, float csy, float csig, float osx, float osy, float osig,
                                             float lo, float hi) {
    const float dcl = sqrtf((lo - csx) * (lo - csx) + csy * csy), dch = sqrtf((hi - csx) * (hi - csx) + csy * csy);
    const float dol = sqrtf((lo - osx) * (lo - osx) + osy * osy), doh = sqrtf((hi - osx) * (hi - osx) + osy * osy);
    const float Dlo = (csig + dcl) - (osig + dol), Dhi = (csig + dch) - (osig + doh);
    // rounding margin: the FP32 copies of s, sigma and the interval ends carry 2^-24
    // relative errors, every evaluated distance a few more; 1e-6 of the sum of magnitudes
    // bounds the error of each difference with ample slack
    const float E = 4.8e-7f * (fabsf(csx) + fabsf(csy) + fabsf(osx) + fabsf(osy) + 2.f * (fabsf(lo) + fabsf(hi)) +
                               csig + osig + dcl + dch + dol + doh) + 1e-30f;
    const bool pos = Dlo > E && Dhi > E, neg = Dlo < -E && Dhi < -E;
    if (!pos && !neg) return CMP_SPLIT;
    if (!(dcl > 0.f && dch > 0.f && dol > 0.f && doh > 0.f)) return CMP_SPLIT;
    // derivative of each distance along the edge: (x - s_x) / |x - s|, increasing in x
    const float gcl = (lo - csx) / dcl, gch = (hi - csx) / dch, gol = (lo - osx) / dol, goh = (hi - osx) / doh;
    const float m0 = gcl - goh - 1e-5f, m1 = gch - gol + 1e-5f;   // D' in [m0, m1]
    const float W = hi - lo;
    if (pos) {
        if (m0 >= 0.f || m1 <= 0.f) return CMP_EXISTING;   // monotone between two positive values
        // min over x of max(Dlo + m0 u, Dhi - m1 (W - u)), u = x - lo in [0, W]
        float u = (Dlo - Dhi + m1 * W) / (m1 - m0);
        u = fminf(fmaxf(u, 0.f), W);
        const float lb = fmaxf(Dlo + m0 * u, Dhi - m1 * (W - u));
        return lb > E ? CMP_EXISTING : CMP_SPLIT;
    }
    if (m0 >= 0.f || m1 <= 0.f) return CMP_CANDIDATE;
    float u = (Dhi - Dlo + m1 * W) / (m1 - m0);   // max over x of min(Dlo + m1 u, Dhi - m0 (W - u))
    u = fminf(fmaxf(u, 0.f), W);
    const float ub = fminf(Dlo + m1 * u, Dhi - m0 * (W - u));
    return ub < -E ? CMP_CANDIDATE : CMP_SPLIT;
}

// Exact split of an overlap [lo, hi] between candidate (a, sa) and existing (b, sb): the
// equal-distance points in FP64, the winner of each piece decided in FP32 when the evaluated
// difference clears its rounding margin, else in FP64 with the exact tie rule (a direct
// window beats one descending from a pseudo-source).  Returns the breakpoints and, per piece,
// whether the candidate wins.
__device__ __noinline__ int split_exact(double ax, double ay, double sa, double bx, double by, double sb, double lo,
                                        double hi, bool c_direct_o_fixed, double* bp, bool* cwin) {
    if (__double_as_longlong(sa) == __double_as_longlong(sb)) {
        // equal path lengths to both pseudo-sources: the candidate is shorter on one side of the
        // perpendicular bisector of a and b, so the overlap splits at most once, at the point
        // where the bisector meets the edge line (x - a_x)^2 + a_y^2 = (x - b_x)^2 + b_y^2
        bp[0] = lo;
        if (ax == bx) {   // D(x) = |x-a| - |x-b| has the sign of |a_y| - |b_y| everywhere
            bp[1] = hi;
            const double d = fabs(ay) - fabs(by);
            cwin[0] = d < 0.0 || (d == 0.0 && c_direct_o_fixed);
            return 1;
        }
        const double xs = 0.5 * (ax + bx) + 0.5 * (by - ay) * (by + ay) / (bx - ax);
        const bool c_left = ax < bx;   // the candidate wins for x < xs iff a_x < b_x
        if (xs > lo && xs < hi) {
            bp[1] = xs; bp[2] = hi;
            cwin[0] = c_left; cwin[1] = !c_left;
            return 2;
        }
        bp[1] = hi;
        cwin[0] = (xs >= hi) ? c_left : !c_left;
        return 1;
    }
    double r0 = 0.0, r1 = 0.0;
    const int nr = equal_points(ax, ay, sa, bx, by, sb, lo, hi, r0, r1);
    bp[0] = lo;
    bp[1] = nr > 0 ? r0 : hi;
    bp[2] = nr > 1 ? r1 : hi;
    bp[nr + 1] = hi;
    const float fax = (float)ax, fay = (float)ay, fsa = (float)sa, fbx = (float)bx, fby = (float)by, fsb = (float)sb;
    const float E = 4.8e-7f * (fabsf(fax) + fabsf(fay) + fabsf(fbx) + fabsf(fby) + 2.f * (fabsf((float)lo) + fabsf((float)hi)) +
                               fsa + fsb) + 1e-30f;
#pragma unroll 1
    for (int q = 0; q < 3; ++q) {
        if (q > nr) break;
        const double xmd = 0.5 * (bp[q] + bp[q + 1]);
        const float xm = (float)xmd;
        const float dcf = fsa + sqrtf((xm - fax) * (xm - fax) + fay * fay);
        const float ddf = dcf - (fsb + sqrtf((xm - fbx) * (xm - fbx) + fby * fby));
        if (fabsf(ddf) > E + 9.6e-7f * dcf) { cwin[q] = ddf < 0.f; continue; }
        const double dc = sa + sqrt((xmd - ax) * (xmd - ax) + ay * ay);
        const double dd = dc - (sb + sqrt((xmd - bx) * (xmd - bx) + by * by));
        const double tie = 1e-13;
        cwin[q] = (dd < -tie * dc) || (dd <= tie * dc && c_direct_o_fixed);
    }
    return nr + 1;
}

// bit-identical pseudo-source and length: the same path family, equal everywhere
template <class R>
__device__ __forceinline__ bool same_family(const Win<R>& a, const Win<R>& b) {
    return __double_as_longlong(a.sx) == __double_as_longlong(b.sx) &&
           __double_as_longlong(a.sy) == __double_as_longlong(b.sy) &&
           __double_as_longlong(a.sig) == __double_as_longlong(b.sig);
}

// Subtract [x0, x1] from a sorted piece list.  Parts narrower than tolw are dropped; a cut
// that would need more than MAXP pieces leaves the piece whole (more coverage, never less).
template <class R>
__device__ __forceinline__ void ivl_sub(Ivl<R>& P, R x0, R x1, R tolw) {
    if (!(x1 > x0)) return;
    Ivl<R> out;
    out.n = 0;
#pragma unroll
    for (int k = 0; k < MAXP; ++k) { out.a[k] = (R)0; out.b[k] = (R)0; }
#pragma unroll 1
    for (int p = 0; p < P.n; ++p) {
        const R a = ivl_get<R>(P.a, p), b = ivl_get<R>(P.b, p);
        const bool l = x0 - a > tolw, r = b - x1 > tolw;
        if (!(x1 > a && x0 < b) || out.n + (l ? 1 : 0) + (r ? 1 : 0) + (P.n - 1 - p) > MAXP) {
            ivl_add<R>(out, a, b);
            continue;
        }
        if (l) ivl_add<R>(out, a, x0);
        if (r) ivl_add<R>(out, x1, b);
    }
    P = out;
}

// Window o (id oi, on the candidate's edge, interval [o0, o1] in the candidate's frame) loses
// the pieces `lost`: it keeps the rest (padded outward by the FP32 widening), in place, as
// extra windows linked right after it, or not at all (then it is marked dead and left in
// the list; the next walk over the list unlinks it).
template <class R, int SH>
__device__ __forceinline__ void window_keep(Ws<R, SH>& ws, WarpSm& sm, const Win<R>& o, int oi, bool same, R o0, R o1,
                                            R Lr, R tolw, const Ivl<R>& lost) {
    Ivl<R> keep;
    keep.n = 0;
#pragma unroll
    for (int k = 0; k < MAXP; ++k) { keep.a[k] = keep.b[k] = (R)0; }
    R cur = o0;
#pragma unroll 1
    for (int q = 0; q < lost.n; ++q) {
        const R l0 = ivl_get<R>(lost.a, q), l1 = ivl_get<R>(lost.b, q);
        if (l0 - cur > tolw) ivl_add<R>(keep, cur, l0);
        if (l1 > cur) cur = l1;
    }
    if (o1 - cur > tolw) ivl_add<R>(keep, cur, o1);
    if (keep.n == 0) {
        ws.win[oi].flags = o.flags & ~WIN_ALIVE;
        return;
    }
    int tail = oi;
    const int onext = ws.win[oi].next;
    const R wpad = (R)Widen<R>::mu * Lr;   // outward rounding of the kept parts
#pragma unroll 1
    for (int q = 0; q < keep.n; ++q) {
        const R ka = ivl_get<R>(keep.a, q), kb = ivl_get<R>(keep.b, q);
        R k0 = (same ? ka : Lr - kb) - wpad;
        R k1 = (same ? kb : Lr - ka) + wpad;
        k0 = k0 < (R)0 ? (R)0 : k0;
        k1 = k1 > Lr ? Lr : k1;
        if (q == 0) { ws.win[oi].b0 = k0; ws.win[oi].b1 = k1; }
        else {
            const int pid = win_alloc<R>(sm, ws.wcap);
            if (pid < 0) break;
            Win<R> piece = o;
            piece.b0 = k0; piece.b1 = k1;
            piece.next = onext;
            ws.win[pid] = piece;
            if (!(o.flags & WIN_DONE)) push_pending<R>(ws, sm, pid, (float)win_key<R>(piece));
            ws.win[tail].next = pid;          // keep the list order
            tail = pid;
        }
    }
}

// Compare candidate c (pseudo-source (csx, csy), length csig, interval [h0, h1] on its
// half-edge che of length Lr) with window o (id oi) of the same edge: on their overlap both
// keep only where they carry the smaller distance.  o's loss is applied at once; the
// candidate's loss (at most three pieces) is returned in cl.
template <class R, int SH>
__device__ __forceinline__ void compare_pair(Ws<R, SH>& ws, WarpSm& sm, int oi, double csx, double csy, double csig,
                                             int che, int cflags, R h0, R h1, R Lr, R tolw, Ivl<R>& cl) {
    cl.n = 0;
#pragma unroll
    for (int k = 0; k < MAXP; ++k) { cl.a[k] = cl.b[k] = (R)0; }
    const Win<R> o = ws.win[oi];
    const bool same = (o.he == che);
    const R o0 = same ? o.b0 : Lr - o.b1, o1 = same ? o.b1 : Lr - o.b0;
    const R lo = h0 > o0 ? h0 : o0, hi = h1 < o1 ? h1 : o1;
    if (!(hi - lo > tolw)) return;
    const bool c_direct = !(cflags & WIN_FIXED);
    Ivl<R> lost;
    lost.n = 0;
#pragma unroll
    for (int k = 0; k < MAXP; ++k) { lost.a[k] = lost.b[k] = (R)0; }
    // FP32 copies of both pseudo-sources in the candidate's frame (conversions in the FP64
    // form; the margins of the FP32 tests cover their rounding)
    const float fcx = (float)csx, fcy = (float)csy, fcs = (float)csig;
    const float fox = same ? (float)fsx(o) : (float)Lr - (float)fsx(o);
    const float foy = same ? (float)fsy(o) : -(float)fsy(o);
    const float fos = (float)fsig(o);
    const bool eq_sig = __double_as_longlong(csig) == __double_as_longlong(o.sig);
    int cmp = CMP_SPLIT;
    if (same && eq_sig && __double_as_longlong(csx) == __double_as_longlong(o.sx) &&
        __double_as_longlong(csy) == __double_as_longlong(o.sy))
        cmp = CMP_EXISTING;   // the same path family: equal everywhere, ties stay
    // the FP32 dominance test (FP64 form only: in the FP32 form it decided too few overlaps to
    // pay for itself on the cutoff workloads, and every overlap goes to the exact split);
    // equal sigma: the exact bisector split below is cheaper than any FP32 attempt
    else if (sizeof(R) == sizeof(double) && !eq_sig) cmp = dominance_f32(fcx, fcy, fcs, fox, foy, fos, (float)lo, (float)hi);
    if (cmp == CMP_EXISTING) ivl_add<R>(cl, lo, hi, false);
    else if (cmp == CMP_CANDIDATE) ivl_add<R>(lost, lo, hi, false);
    else {
        // split of the overlap at the equal-distance points (FP64 roots in both forms; an
        // FP32 attempt with rigorous margins decided too few splits to pay for its code)
        R bq[4];
        bool cw[3];
        const double Ld = (double)Lr;
        const double osx = same ? o.sx : Ld - o.sx, osy = same ? o.sy : -o.sy;
        double bp[4];
        const int npz = split_exact(csx, csy, csig, osx, osy, o.sig, (double)lo, (double)hi,
                                    c_direct && (o.flags & WIN_FIXED), bp, cw);
        bq[0] = (R)bp[0]; bq[1] = (R)bp[1]; bq[2] = (R)bp[2]; bq[3] = (R)bp[3];
#pragma unroll 1
        for (int q = 0; q < npz; ++q) {
            if (cw[q]) ivl_add<R>(lost, bq[q], bq[q + 1], false);
            else ivl_add<R>(cl, bq[q], bq[q + 1], false);
        }
    }
    if (lost.n > 0) window_keep<R>(ws, sm, o, oi, same, o0, o1, Lr, tolw, lost);
}

// Windows a lane collects per walk of an insertion round.
constexpr int WALK_K = 4;

// One insertion round, all lanes together.  Lane l (has) inserts candidate c into the list
// of edge slot es; lanes of one round hold different edges.  A candidate on an empty edge
// is linked at once.  The others alternate walks and comparisons until their lists are
// done: each lane walks its list (unlinking dead windows) and collects up to WALK_K live
// windows overlapping its candidate's hull; the collected (candidate, window) pairs are
// spread over all 32 lanes, each compares one pair, applies the window's loss, and hands the
// candidate's loss back to its lane, which cuts it from the candidate's pieces.  Every window
// on an edge is compared with the whole candidate; the candidate keeps the points where it
// beats all of them, and each window the points where the candidate does not beat it, so
// the smallest distance at every point stays covered.  What remains of the candidate is
// linked at the head of the list.
template <class R, int SH>
__device__ __noinline__ void insert_round(const DMesh& m, Ws<R, SH>& ws, WarpSm& sm, bool has, int es,
                                          const Win<R>& c0, double rc, int lane) {
    Win<R> c = c0;
    R Lr = (R)0, tolw = (R)0;
    int cursor = -1;
    if (has) {
        Lr = sizeof(R) == sizeof(float) ? (R)m.he32[c.he].L : (R)m.he[c.he].L;
        tolw = (R)Tol<R>::w * Lr;
        if (c.b0 < (R)0) c.b0 = (R)0;
        if (c.b1 > Lr) c.b1 = Lr;
        has = (c.b1 - c.b0 > tolw) && (double)win_key<R>(c) < rc;
        if (has) cursor = ws.ehead[es];
        c.flags = (c.flags & WIN_FIXED) | WIN_ALIVE;
    }
    if (has && cursor < 0) {   // first window on this edge: nothing to intersect with
        has = false;
        const int id = win_alloc<R>(sm, ws.wcap);
        if (id >= 0) {
            c.next = -1;
            ws.win[id] = c;
            ws.ehead[es] = id;
            push_pending<R>(ws, sm, id, (float)win_key<R>(c));
            face_add(ws, sm, c.he / 3);
        }
    }
    if (!__any_sync(CSS_FULL, has)) return;
    Ivl<R> pc;
    pc.n = has ? 1 : 0;
    pc.a[0] = c.b0; pc.b[0] = c.b1;
#pragma unroll
    for (int k = 1; k < MAXP; ++k) { pc.a[k] = (R)0; pc.b[k] = (R)0; }
    int prev = -1, guard = 0, err = 0;
    while (__any_sync(CSS_FULL, has && cursor >= 0 && pc.n > 0)) {
        // ---- walk: up to WALK_K live windows overlapping the candidate's hull
        int ids[WALK_K];
#pragma unroll
        for (int k = 0; k < WALK_K; ++k) ids[k] = -1;
        int n = 0;
        const R h0 = pc.n > 0 ? ivl_get<R>(pc.a, 0) : (R)0, h1 = pc.n > 0 ? ivl_get<R>(pc.b, pc.n - 1) : (R)0;
        if (has && pc.n > 0) {
            // windows split by the last comparisons sit between prev and cursor
            if (prev >= 0) {
                int x = ws.win[prev].next;
                while (x >= 0 && x != cursor && guard <= ws.wcap) { prev = x; x = ws.win[x].next; ++guard; }
            }
            while (cursor >= 0 && n < WALK_K) {
                if (++guard > ws.wcap) { err |= css::ST_ITER_LIMIT; cursor = -1; break; }
                const Win<R> o = ws.win[cursor];
                if (!(o.flags & WIN_ALIVE)) {                 // unlink dead windows
                    if (prev < 0) ws.ehead[es] = o.next; else ws.win[prev].next = o.next;
                    cursor = o.next;
                    continue;
                }
                const bool same = (o.he == c.he);
                const R o0 = same ? o.b0 : Lr - o.b1, o1 = same ? o.b1 : Lr - o.b0;
                const R lo = h0 > o0 ? h0 : o0, hi = h1 < o1 ? h1 : o1;
                if (hi - lo > tolw) { reg_set(ids, n, cursor); ++n; }
                prev = cursor;
                cursor = o.next;
            }
        }
        // ---- the pairs of all lanes, dense in lane order
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(CSS_FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(CSS_FULL, incl, 31);
        const int excl = incl - n;
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            int owner = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int v = __shfl_sync(CSS_FULL, incl, owner + step - 1);
                if (v <= t) owner += step;
            }
            owner = min(owner, 31);
            const int j = t - __shfl_sync(CSS_FULL, excl, owner);
            int oi = -1;
#pragma unroll
            for (int k = 0; k < WALK_K; ++k) {
                const int v = __shfl_sync(CSS_FULL, ids[k], owner);
                if (k == j) oi = v;
            }
            const double csx = __shfl_sync(CSS_FULL, c.sx, owner), csy = __shfl_sync(CSS_FULL, c.sy, owner);
            const double csig = __shfl_sync(CSS_FULL, c.sig, owner);
            const int che = __shfl_sync(CSS_FULL, c.he, owner), cfl = __shfl_sync(CSS_FULL, c.flags, owner);
            const R ch0 = __shfl_sync(CSS_FULL, h0, owner), ch1 = __shfl_sync(CSS_FULL, h1, owner);
            const R cL = __shfl_sync(CSS_FULL, Lr, owner), ctol = __shfl_sync(CSS_FULL, tolw, owner);
            Ivl<R> cl;
            cl.n = 0;
#pragma unroll
            for (int k = 0; k < MAXP; ++k) { cl.a[k] = cl.b[k] = (R)0; }
            if (t < total && oi >= 0) compare_pair<R>(ws, sm, oi, csx, csy, csig, che, cfl, ch0, ch1, cL, ctol, cl);
            // each lane takes back its pairs' losses from the lanes that compared them (a
            // comparison's loss is at most two pieces: the winners of its sub-intervals
            // alternate once the touching ones are merged)
#pragma unroll 1
            for (int k = 0; k < WALK_K; ++k) {
                const int src = excl + k - t0;
                const bool in = k < n && src >= 0 && src < 32;
                const int s = in ? src : lane;
                const int nl = __shfl_sync(CSS_FULL, cl.n, s);
#pragma unroll 1
                for (int r = 0; r < 2; ++r) {
                    const R x0 = __shfl_sync(CSS_FULL, ivl_get<R>(cl.a, r), s);
                    const R x1 = __shfl_sync(CSS_FULL, ivl_get<R>(cl.b, r), s);
                    if (in && r < nl) ivl_sub<R>(pc, x0, x1, tolw);
                }
            }
        }
        __syncwarp();
    }
    if (err) atomicOr(&sm.err, err);
    bool added = false;
#pragma unroll 1
    for (int p = 0; p < pc.n; ++p) {
        Win<R> w = c;
        w.b0 = ivl_get<R>(pc.a, p);
        w.b1 = ivl_get<R>(pc.b, p);
        if (!((double)win_key<R>(w) < rc)) continue;
        const int id = win_alloc<R>(sm, ws.wcap);
        if (id < 0) break;
        w.next = ws.ehead[es];
        ws.win[id] = w;
        ws.ehead[es] = id;
        push_pending<R>(ws, sm, id, (float)win_key<R>(w));
        added = true;
    }
    if (added) face_add(ws, sm, c.he / 3);
}

// ------------------------------------------------------------------ warp-cooperative rounds
__device__ __forceinline__ int group_rounds(bool has, int key, int lane, int& rank) {
    const int k = has ? key : (-1 - lane);
    const unsigned grp = __match_any_sync(CSS_FULL, k);
    rank = __popc(grp & css::lanemask_lt());
    return (int)__reduce_max_sync(CSS_FULL, (unsigned)__popc(grp));
}

// Vertex table flags: bit 0 queued for emission, bit 1 distance from a pseudo-source path,
// bits 16..31 the back direction of the recorded path (DMesh::cang units) in steps of 1/4096
// rad offset by 4 rad; 0xffff where it is unknown or out of range.
constexpr float BACK_STEP = 4096.0f, BACK_OFF = 4.0f;
__device__ __forceinline__ unsigned pack_back(float b) {
    const float t = (b + BACK_OFF) * BACK_STEP;
    return (t >= 0.0f && t < 65535.0f) ? (unsigned)__float2int_rn(t) : 0xffffu;   // NaN -> unknown
}

template <class R, int SH>
__device__ __noinline__ void vertex_round(const DMesh& m, Ws<R, SH>& ws, WarpSm& sm, bool has,
                                          const VCand<R, SH == 2>& c, double rc, int lane) {
    if (!__any_sync(CSS_FULL, has)) return;
    bool claimed = false;
    int slot = -1;
    if (has) {
        slot = ws_vins<R>(ws, c.v, claimed);
        if (slot < 0) { atomicOr(&sm.err, css::ST_HASH_OVERFLOW); has = false; }
    }
    if (claimed) {
        ws.vdist[slot] = __longlong_as_double(0x7ff0000000000000ll);
        ws.vflag[slot] = 0;
        if (!ws.shared) ws.vvid[slot] = c.v;
    }
    __syncwarp();
    int rank;
    const int rounds = group_rounds(has, slot, lane, rank);
    for (int q = 0; q < rounds; ++q) {
        if (has && rank == q) {
            const double d = c.d;
            const double vd = ws.vdist[slot];
            const int vf = ws.vflag[slot];
            const double tie = 1e-13 * d;    // lengths are exact FP64 here in both forms
            // shorter beyond rounding, or a tie won by a direct path over a pseudo-source one
            if (d < vd - tie || (d <= vd + tie && !c.fixed && (vf & 2))) {
                ws.vdist[slot] = d < vd ? d : vd;
                ws.vtan[2 * slot] = c.tx;
                ws.vtan[2 * slot + 1] = c.ty;
                ws.vflag[slot] = (int)((pack_back(c.back) << 16) | (unsigned)(c.fixed ? ((vf | 2) & 3) : (vf & 1)));
                if constexpr (SH == 2) {
                    ws.lpar[slot] = c.par;
                    ws.lfk[slot] = c.fk;
                    ws.ldir[2 * slot] = c.dx;
                    ws.ldir[2 * slot + 1] = c.dy;
                    ws.llen[slot] = c.len;
                }
                if (d < vd && d < rc) atomicMin(&sm.emin, __float_as_uint(__double2float_rd(d)));
                if (d < vd && d < rc && !(ws.vflag[slot] & 1)) {
                    ws.vflag[slot] |= 1;
                    const int p = atomicAdd(&sm.nemit, 1);
                    if (p < ws.emcap) ws.emit[p] = slot;
                    else atomicOr(&sm.err, css::ST_HASH_OVERFLOW);
                }
            }
        }
        __syncwarp();
    }
}

// Children on one edge go in one at a time.  With a carry buffer (room for 32, its fill
// count at ncar), the second and later ones on an edge wait there for the next wave's rounds
// instead of taking rounds of their own now (most of such a round's lanes would idle); their
// smallest key joins the bound below which vertices may emit, since their candidates are at
// least that key.
constexpr int CARRY_CAP = 32;
template <class R, int SH>
__device__ __noinline__ void child_round(const DMesh& m, Ws<R, SH>& ws, WarpSm& sm, bool has, const Win<R>& c, double rc,
                                         int lane, Win<R>* carry = nullptr, int* ncar = nullptr) {
    if (!__any_sync(CSS_FULL, has)) return;
    bool claimed = false;
    int slot = -1;
    if (has) {
        slot = ws_eins<R>(ws, m.edge[c.he], claimed);
        if (slot < 0) { atomicOr(&sm.err, css::ST_HASH_OVERFLOW); has = false; }
    }
    if (claimed) ws.ehead[slot] = -1;
    __syncwarp();
    int rank;
    int rounds = group_rounds(has, slot, lane, rank);
    if (carry && rounds > 1) {
        const unsigned later = __ballot_sync(CSS_FULL, has && rank > 0);
        const int n0 = *ncar;
        if (n0 + __popc(later) <= CARRY_CAP) {
            if (has && rank > 0) {
                carry[n0 + __popc(later & css::lanemask_lt())] = c;
                atomicMin(&sm.cmin, __float_as_uint(__double2float_rd((double)win_key<R>(c))));
                has = false;
            }
            __syncwarp();
            if (lane == 0) *ncar = n0 + __popc(later);
            rounds = 1;
        }
    }
    for (int q = 0; q < rounds; ++q) {
        insert_round<R>(m, ws, sm, has && rank == q, slot, c, rc, lane);
        __syncwarp();
    }
}

// Pseudo-source vertices whose distance is final start windows on the edges opposite
// them; those one-ring faces join the target faces (paths may bend there, Sec. 2.2).  A
// vertex's distance is final once no queued window can still shorten it: every
// candidate a window yields is at least that window's key, so vertices with
// d(v) <= kmin (the smallest queued key) go now and the others wait.  Returns the number
// of vertices emitted.
// Only corners that meet the vertex's shadow get a window: a shortest path that passes
// through an interior vertex of angle sum T leaves it at least pi away from its incoming
// direction on both sides, i.e. within [b + pi, b + T - pi] of the back direction b of any
// shortest path to the vertex (outside that range the bend can be cut short on the side
// where it is below pi, so the continuation is not shortest).  The range is widened by
// SHADOW_TOL for the rounding of b and of the corner angles; vertices without a known back
// direction, boundary and non-manifold vertices emit on every corner.
constexpr float SHADOW_TOL = 1e-3f;
template <class R, int SH>
__device__ __noinline__ int emit_round(const DMesh& m, Ws<R, SH>& ws, WarpSm& sm, double rc, double kmin, int lane,
                                       Win<R>* stage = nullptr, int cap = 0, int* nstaged = nullptr) {
    __syncwarp();
    int staged = 0;   // windows handed to the caller in stage (team form) instead of inserted
    const int ne = min(sm.nemit, ws.emcap);
    if (ne == 0) return 0;
    // the vertices that wait are compacted to the front of the list in place (a write
    // never lands behind the entries still to be read)
    int n_wait = 0;
    int emitted = 0;
    float wmin = INFINITY;   // smallest distance among the vertices left waiting
    for (int base = 0; base < ne; base += 32) {
        const int it = base + lane;
        int vs = -1;
        bool go = false;
        if (it < ne) {
            vs = ws.emit[it];
            const double dv0 = ws.vdist[vs];
            go = dv0 <= kmin;
            if (!go) wmin = fminf(wmin, __double2float_rd(dv0));
        }
        __syncwarp();
        const unsigned gm = __ballot_sync(CSS_FULL, go);
        const unsigned wm = __ballot_sync(CSS_FULL, it < ne && !go);
        if (it < ne && !go) ws.emit[n_wait + __popc(wm & css::lanemask_lt())] = vs;
        n_wait += __popc(wm);
        // emit this chunk's vertices now (at most 32)
        const bool has = go;
        int vid = 0, rs = 0, len = 0;
        double dv = 0.0;
        R tx = (R)0, ty = (R)0;
        float lo = -INFINITY, hi = INFINITY, th = 0.0f;   // the shadow, [lo, hi] (mod th)
        if (has) {
            vid = ws.vvid[vs];
            dv = ws.vdist[vs];
            tx = ws.vtan[2 * vs];
            ty = ws.vtan[2 * vs + 1];
            const int fl = ws.vflag[vs];
            ws.vflag[vs] = fl & ~1;
            rs = m.ring_start[vid];
            len = m.ring_start[vid + 1] - rs;
            const unsigned qb = (unsigned)fl >> 16;
            if (qb != 0xffffu) {
                th = (float)m.theta[vid];
                const float b = (float)qb * (1.0f / BACK_STEP) - BACK_OFF;
                lo = b + 3.14159265f - SHADOW_TOL;
                lo -= th * floorf(lo / th);
                hi = lo + (th - 6.28318531f + 2.0f * SHADOW_TOL);
            }
        }
        // one window per (emitting vertex, opposite edge), 32 at a time: lane t takes the
        // t-th pair of the flattened list (owner = the vertex whose ring holds it)
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(CSS_FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(CSS_FULL, incl, 31);
        for (int tb = 0; tb < total; tb += 32) {
            const int t = tb + lane;
            int owner = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int v = __shfl_sync(CSS_FULL, incl, owner + step - 1);
                if (v <= t) owner += step;
            }
            owner = min(owner, 31);
            const int o_rs = __shfl_sync(CSS_FULL, rs, owner);
            const int o_ex = __shfl_sync(CSS_FULL, incl - len, owner);
            const double o_dv = __shfl_sync(CSS_FULL, dv, owner);
            const R o_tx = __shfl_sync(CSS_FULL, tx, owner);
            const R o_ty = __shfl_sync(CSS_FULL, ty, owner);
            const float o_lo = __shfl_sync(CSS_FULL, lo, owner);
            const float o_hi = __shfl_sync(CSS_FULL, hi, owner);
            const float o_th = __shfl_sync(CSS_FULL, th, owner);
            int o_vid = 0;
            if constexpr (SH == 2) o_vid = __shfl_sync(CSS_FULL, vid, owner);
            bool hh = t < total;
            Win<R> c;
            if (hh) {
                const int hc = m.ring[o_rs + (t - o_ex)];
                const int f = hc / 3, k = hc - 3 * f;
                const int hop = 3 * f + (k == 2 ? 0 : k + 1);
                // the corner's wedge [a, a + w] against the shadow, one turn either way; NaN
                // bounds never miss.  A corner outside the shadow adds neither a window nor its
                // face: no shortest path leaves the vertex into it
                const float2 cw = m.cang[hc];
                bool miss = true;
#pragma unroll 1
                for (int s = -1; s <= 1; ++s) {
                    const float a = cw.x + (float)s * o_th;
                    if (!(a > o_hi || a + cw.y < o_lo)) miss = false;
                }
                if (!miss) face_add(ws, sm, f);
                const int tw = miss ? -1 : m.twin[hop];
                if (tw < 0) hh = false;
                else {
                    const HeRec r = m.he[hop];
                    c.he = tw;
                    c.b0 = (R)0;
                    c.b1 = (R)r.L;
                    c.sx = r.L - r.cx;
                    c.sy = -r.cy;
                    c.sig = o_dv;
                    set_fast(c);
                    c.ta = o_tx;
                    c.tb = o_ty;
                    c.flags = WIN_FIXED | WIN_ALIVE;
                    c.next = -1;
                    if constexpr (SH == 2) c.pv = o_vid;
                }
            }
            if (stage) {   // the team inserts these together; what does not fit is inserted here
                const unsigned hm = __ballot_sync(CSS_FULL, hh);
                if (staged + __popc(hm) <= cap) {
                    if (hh) stage[staged + __popc(hm & css::lanemask_lt())] = c;
                    staged += __popc(hm);
                    continue;
                }
            }
            child_round<R>(m, ws, sm, hh, c, rc, lane);
        }
        emitted += __popc(gm);
    }
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wmin = fminf(wmin, __shfl_xor_sync(CSS_FULL, wmin, o));
    if (lane == 0) {
        sm.nemit = n_wait;   // inserting windows never touches the vertex list
        sm.emin = __float_as_uint(wmin);
        if (nstaged) *nstaged = staged;
    }
    __syncwarp();
    return emitted;
}

__device__ __forceinline__ double pot_dudl(const css_potential& p, double l) {
    if (!(l < p.r_cut)) return 0.0;
    if (p.kind == CSS_POT_HARMONIC) return -2.0 * p.eps * (1.0 - l / p.sigma) / p.sigma;
    if (p.kind == CSS_POT_WCA) {
        const double q = p.sigma / l, q2 = q * q, q6 = q2 * q2 * q2;
        return 24.0 * p.eps * (q6 - 2.0 * q6 * q6) / l;
    }
    return -(l / (p.sigma * p.sigma)) * p.A * exp(-l * l / (2.0 * p.sigma * p.sigma));
}

__device__ __forceinline__ double pot_u(const css_potential& p, double l) {
    if (!(l < p.r_cut)) return 0.0;
    if (p.kind == CSS_POT_HARMONIC) { const double u = 1.0 - l / p.sigma; return p.eps * u * u; }
    if (p.kind == CSS_POT_WCA) {
        const double q = p.sigma / l, q2 = q * q, q6 = q2 * q2 * q2;
        return 4.0 * p.eps * (q6 * q6 - q6) + p.eps;
    }
    return p.A * exp(-l * l / (2.0 * p.sigma * p.sigma));
}

// distance + source tangent (source-face layout) of particle j of face fl
template <class R, int SH>
__device__ __noinline__ double query(const DMesh& m, const Ws<R, SH>& ws, int f0, R qx, R qy, int fl, const double* bj,
                                     R& tx, R& ty, VLink<SH == 2>* ql) {
    R L01, x2, y2, dummy;
    face_corner_f<R>(m, fl, 1, L01, dummy);
    face_corner_f<R>(m, fl, 2, x2, y2);
    const R b1 = (R)bj[1], b2 = (R)bj[2];
    const R px = b1 * L01 + b2 * x2, py = b2 * y2;
    double best = __longlong_as_double(0x7ff0000000000000ll);
    bool best_fixed = true;
    const double tie = Tie<R>::rel;
    // FP32 form: candidates within the FP32 band of the current best are re-compared with
    // exact FP64 lengths (near-degenerate predicate); best_exact holds the best's FP64 length
    double best_exact = best;
    tx = (R)0; ty = (R)0;
    if constexpr (SH == 2) { ql->par = -1; ql->fk = 4 * fl + 3; ql->dx = 1.0; ql->dy = 0.0; ql->len = 0.0; }
    if (fl == f0) {
        const R dx = px - qx, dy = py - qy;
        const R d = sqrt(dx * dx + dy * dy);
        best = (double)d;
        best_exact = best;
        best_fixed = false;
        if (d > (R)0) { tx = dx / d; ty = dy / d; }
        if constexpr (SH == 2) {   // straight back to the source
            ql->dx = d > (R)0 ? -(double)tx : 1.0;
            ql->dy = d > (R)0 ? -(double)ty : 0.0;
            ql->len = (double)d;
        }
    }
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
        const int h = 3 * fl + k;
        const int slot = ws_efind<R>(ws, m.edge[h]);
        if (slot < 0) continue;
        R ax, ay, bx, by;
        face_corner_f<R>(m, fl, k, ax, ay);
        face_corner_f<R>(m, fl, k + 1, bx, by);
        R L;
        if (sizeof(R) == sizeof(float)) L = (R)m.he32[h].L; else L = (R)m.he[h].L;
        const R dx = (bx - ax) / L, dy = (by - ay) / L;
        const R hx = (px - ax) * dx + (py - ay) * dy;
        const R hy = dx * (py - ay) - dy * (px - ax);
        // FP32 form: the target in this edge's frame from the FP64 layout, for exact lengths in
        // near-ties (computed once per edge)
        double hxd = 0.0, hyd = 0.0;
        if (sizeof(R) == sizeof(float)) {
            double axd, ayd, bxd, byd;
            css::face_corner(m, fl, k, axd, ayd);
            css::face_corner(m, fl, k + 1, bxd, byd);
            const double Ldd = m.he[h].L;
            const double pxd = bj[1] * m.lay[3 * fl] + bj[2] * m.lay[3 * fl + 1], pyd = bj[2] * m.lay[3 * fl + 2];
            const double ddx = (bxd - axd) / Ldd, ddy = (byd - ayd) / Ldd;
            hxd = (pxd - axd) * ddx + (pyd - ayd) * ddy;
            hyd = ddx * (pyd - ayd) - ddy * (pxd - axd);
        }
        // cone tolerance of the interval precision: adjacent windows stored in FP32 may
        // leave or overlap by an ulp of the edge length, which must not hide a target
        const R tol = (R)Tol<R>::w * L;
        int guard = 0;
        for (int wi = ws.ehead[slot]; wi >= 0 && guard < ws.wcap; ++guard) {
            const Win<R> w = ws.win[wi];
            wi = w.next;
            if (!(w.flags & WIN_ALIVE) || w.he != h) continue;
            bool inside;
            if (win_degen<R>(w, L)) inside = win_degen_sees<R>(w, L);
            else {
                const R X = fsx(w) + (hx - fsx(w)) * (-fsy(w)) / (hy - fsy(w));
                inside = X >= w.b0 - tol && X <= w.b1 + tol;
            }
            if (!inside) continue;
            double d = (double)win_dist<R>(w, hx, hy);
            const bool direct = !(w.flags & WIN_FIXED);
            double t_tie = tie;
            double cmp_best = best;
            if (sizeof(R) == sizeof(float) && fabs(d - best) <= 1e-5 * d) {
                d = win_dist_exact<R>(w, hxd, hyd);   // exact lengths near a tie
                cmp_best = best_exact;
                t_tie = 1e-13;
            }
            if (d < cmp_best - t_tie * d || (d <= cmp_best + t_tie * d && direct && best_fixed)) {
                best = d < cmp_best ? d : cmp_best;
                best_exact = sizeof(R) == sizeof(float) ? win_dist_exact<R>(w, hxd, hyd) : d;
                best_fixed = !direct;
                win_tangent<R>(w, hx, hy, tx, ty);
                if constexpr (SH == 2) {
                    win_link(m, w, hx, hy, -1, *ql);
                    ql->fk = 4 * fl + 3;
                }
            }
        }
    }
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
        const int32_t v = m.fv[3 * fl + k];
        if (!m.pseudo[v]) continue;   // only pseudo-source vertices can bend a shortest path
        const int slot = ws_vfind<R>(ws, v);
        if (slot < 0) continue;
        R vx, vy;
        face_corner_f<R>(m, fl, k, vx, vy);
        const double d = ws.vdist[slot] + (double)sqrt((px - vx) * (px - vx) + (py - vy) * (py - vy));
        if (d < best - tie * d) {
            best = d; best_exact = d; best_fixed = true; tx = ws.vtan[2 * slot]; ty = ws.vtan[2 * slot + 1];
            if constexpr (SH == 2) {   // straight to the vertex, then along its path
                const double ex = (double)(vx - px), ey = (double)(vy - py), n = sqrt(ex * ex + ey * ey);
                ql->par = v;
                ql->fk = 4 * fl + 3;
                ql->dx = n > 0.0 ? ex / n : 1.0;
                ql->dy = n > 0.0 ? ey / n : 0.0;
                ql->len = n;
            }
        }
    }
    return best;
}

// Smallest and largest queued key.
template <class R, int SH>
__device__ __forceinline__ void pending_range(const Ws<R, SH>& ws, int npend, int lane, float& kmin, float& kmax) {
    kmin = INFINITY;
    kmax = 0.0f;
    for (int i = lane; i < npend; i += 32) {
        const float k = ws.pk[i];
        kmin = fminf(kmin, k);
        kmax = fmaxf(kmax, k);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = fminf(kmin, __shfl_xor_sync(CSS_FULL, kmin, o));
        kmax = fmaxf(kmax, __shfl_xor_sync(CSS_FULL, kmax, o));
    }
}

// The next wave: up to 32 queued windows among those with the smallest keys.  A key
// threshold T is bisected until 32..64 queued keys lie at or below it; the first 32 of
// those in queue order are taken and the queue is compacted in place.  Processing in
// (batched) key order keeps the work close to that of a priority queue: windows that a
// shorter family would trim are mostly never unfolded.
template <class R, int SH>
__device__ int select_wave(Ws<R, SH>& ws, WarpSm& sm, int npend, float kmin, float kmax, int lane) {
    float T = kmax;
    if (npend > 32) {
        float lo = kmin, hi = kmax;
        for (int it = 0; it < 12; ++it) {
            const float mid = 0.5f * (lo + hi);
            if (!(mid > lo && mid < hi)) break;
            int c = 0;
            for (int i = lane; i < npend; i += 32) c += ws.pk[i] <= mid ? 1 : 0;
            c = (int)__reduce_add_sync(CSS_FULL, (unsigned)c);
            if (c < 32) lo = mid;
            else {
                hi = mid;
                T = mid;
                if (c <= 64) break;
            }
        }
    }
    int taken = 0, kept = 0;
    for (int base = 0; base < npend; base += 32) {
        const int i = base + lane;
        int id = -1;
        float k = 0.0f;
        if (i < npend) { id = ws.pq[i]; k = ws.pk[i]; }
        __syncwarp();
        const bool cand = i < npend && k <= T;
        const unsigned cm = __ballot_sync(CSS_FULL, cand);
        const int r = taken + __popc(cm & css::lanemask_lt());
        const bool take = cand && r < 32;
        const bool keep = i < npend && !take;
        const unsigned km = __ballot_sync(CSS_FULL, keep);
        if (take) sm.sel[r] = id;
        if (keep) {   // kept entries move forward only: p <= i
            const int p = kept + __popc(km & css::lanemask_lt());
            ws.pq[p] = id;
            ws.pk[p] = k;
        }
        taken = min(32, taken + __popc(cm));
        kept += __popc(km);
    }
    __syncwarp();
    const int mine = lane < taken ? sm.sel[lane] : -1;
    __syncwarp();
    if (lane == 0) sm.npend = kept;
    __syncwarp();
    return mine;
}

// Start a source: empty tables and counters, the source's face, distance candidates for its
// pseudo-source corners and one window per edge of its face covering the whole edge (run by
// one warp).
template <class R, int SH>
__device__ __forceinline__ void seed_source(const DMesh& m, Ws<R, SH>& ws, WarpSm& sm, int f0, double qxd, double qyd,
                                            double rc, int lane) {
    ws_clear_shared<R>(ws, lane);
    if (lane == 0) { sm.nwin = 0; sm.npend = 0; sm.nface = 0; sm.nemit = 0; sm.err = 0; sm.emin = 0x7f800000u; sm.ncar = 0; sm.cmin = 0x7f800000u; }
    __syncwarp();
    if (lane == 0) face_add(ws, sm, f0);
    {   // the source's own pseudo-source corners
        VCand<R, SH == 2> c;
        bool has = false;
        if (lane < 3) {
            c.v = m.fv[3 * f0 + lane];
            has = m.pseudo[c.v] != 0;
            double vx, vy;
            css::face_corner(m, f0, lane, vx, vy);
            const double dx = vx - qxd, dy = vy - qyd, d = sqrt(dx * dx + dy * dy);
            c.fixed = 0;
            c.d = d;
            c.tx = (R)(d > 0.0 ? dx / d : 1.0);
            c.ty = (R)(d > 0.0 ? dy / d : 0.0);
            double nx, ny;   // the corner's first edge runs to the next corner of the face
            css::face_corner(m, f0, lane + 1, nx, ny);
            c.back = back_angle(m, 3 * f0 + lane, nx - vx, ny - vy, -dx, -dy, m.lay[3 * f0]);
            if constexpr (SH == 2) {   // straight back to the source
                c.par = -1;
                c.fk = 4 * f0 + lane;
                c.dx = d > 0.0 ? -dx / d : -1.0;
                c.dy = d > 0.0 ? -dy / d : 0.0;
                c.len = d;
            }
        }
        vertex_round<R>(m, ws, sm, has, c, rc, lane);
    }
    {   // one window per edge of the source face, covering the whole edge
        Win<R> c;
        bool has = false;
        if (lane < 3) {
            const int h = 3 * f0 + lane;
            const int tw = m.twin[h];
            if (tw >= 0) {
                has = true;
                double ax, ay, bx, by;
                css::face_corner(m, f0, lane, ax, ay);
                css::face_corner(m, f0, lane + 1, bx, by);
                const double L = m.he[h].L;
                const double dx = (bx - ax) / L, dy = (by - ay) / L;
                const double hx = (qxd - ax) * dx + (qyd - ay) * dy;
                const double hy = dx * (qyd - ay) - dy * (qxd - ax);
                c.he = tw;
                c.b0 = (R)0;
                c.b1 = (R)m.he[tw].L;
                c.sx = L - hx;
                c.sy = hy > 0.0 ? -hy : 0.0;
                c.sig = 0.0;
                set_fast(c);
                c.ta = (R)(-dx);
                c.tb = (R)dy;
                c.flags = WIN_ALIVE;
                c.next = -1;
                if constexpr (SH == 2) c.pv = -1;
            }
        }
        child_round<R>(m, ws, sm, has, c, rc, lane);
    }
}

// One chunk of targets (one warp): lane l evaluates particle j in face fl if has: its distance
// and tangent at the source, its pair row entry (slots(ballot of pairs) gives where this
// chunk's pairs start in the row) and its force and energy terms.
template <class R, int SH, class Slots>
__device__ __forceinline__ void eval_targets(const cssi::GeoJob& J, int i, const Ws<R, SH>& ws, int f0, R qx, R qy,
                                             bool has, int o_fl, int j, int lane, int item, Slots slots, double& fx,
                                             double& fy, double& en) {
    const DMesh& m = J.m;
    const double rc = J.rc;
    const bool wp = J.want_pairs != 0;
    bool ispair = false;
    double d = 0.0;
    R tx = (R)0, ty = (R)0;
    VLink<SH == 2> ql;
    if (has) {
        d = query<R>(m, ws, f0, qx, qy, o_fl, J.bary + 3 * (size_t)j, tx, ty, &ql);
        ispair = d < rc;
    }
    const unsigned pm = __ballot_sync(CSS_FULL, ispair);
    const int pbase = slots(pm);   // the row slots of this chunk's pairs start here
    if constexpr (SH == 2) {
        // the pair's legs, from the target back to the source: its own link, then the
        // link of each vertex on the way (still in this source's table)
        const int pos = pbase + __popc(pm & css::lanemask_lt());
        if (ispair && pos < J.pair_cap) {
            const size_t o = (size_t)item * J.pair_cap + pos;
            int nl = 0;
            VLink<true> l = ql;
            for (;;) {
                if (nl >= J.lmax) { nl = -1; break; }
                const size_t a = o * J.lmax + nl;
                J.lfk[a] = l.fk;
                J.ldir[2 * a] = l.dx;
                J.ldir[2 * a + 1] = l.dy;
                J.llen[a] = l.len;
                ++nl;
                if (l.par < 0) break;
                const int slot = ws_vfind<R>(ws, l.par);
                if (slot < 0) { nl = -2; break; }
                l.par = ws.lpar[slot];
                l.fk = ws.lfk[slot];
                l.dx = ws.ldir[2 * slot];
                l.dy = ws.ldir[2 * slot + 1];
                l.len = ws.llen[slot];
            }
            J.lnum[o] = nl;
        }
    }
    if (wp && ispair) {
        const int pos = pbase + __popc(pm & css::lanemask_lt());
        if (pos < J.pair_cap) {
            const size_t o = (size_t)i * J.pair_cap + pos;
            J.pj[o] = j;
            J.pd[o] = d;
            const double* fr = m.frame + 9 * (size_t)f0;
            J.pt[3 * o] = (double)tx * fr[3] + (double)ty * fr[6];
            J.pt[3 * o + 1] = (double)tx * fr[4] + (double)ty * fr[7];
            J.pt[3 * o + 2] = (double)tx * fr[5] + (double)ty * fr[8];
        }
    }
    if (ispair && J.want_forces) {
        const double du = pot_dudl(J.pot, d);
        fx += du * (double)tx;
        fy += du * (double)ty;
        en += 0.5 * pot_u(J.pot, d);
    }
}

// The targets in the faces flist[fb .. fb + 32) (one warp): each particle's distance and
// tangent at the source, its pair row entry (slots(ballot of pairs) gives where this chunk's
// pairs start in the row) and its force and energy terms.
template <class R, int SH, class Slots>
__device__ __forceinline__ void eval_face_block(const cssi::GeoJob& J, int i, const Ws<R, SH>& ws, int f0, R qx, R qy,
                                                int fb, int nface, int lane, int item, Slots slots, double& fx,
                                                double& fy, double& en) {
    const DMesh& m = J.m;
    const int fi = fb + lane;
    int fl = -1, st = 0, cnt = 0;
    if (fi < nface) {
        fl = ws.flist[fi];
        const int key = m.frank ? m.frank[fl] : fl;
        st = J.fstart[key];
        cnt = J.fstart[key + 1] - st;
    }
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(CSS_FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(CSS_FULL, incl, 31);
    for (int tb = 0; tb < total; tb += 32) {
        const int t = tb + lane;
        int owner = 0;
        for (int step = 16; step >= 1; step >>= 1) {
            const int v = __shfl_sync(CSS_FULL, incl, owner + step - 1);
            if (v <= t) owner += step;
        }
        owner = min(owner, 31);
        const int o_fl = __shfl_sync(CSS_FULL, fl, owner);
        const int o_st = __shfl_sync(CSS_FULL, st, owner);
        const int o_ex = __shfl_sync(CSS_FULL, incl - cnt, owner);
        int j = -1;
        if (t < total) j = J.fitems[o_st + (t - o_ex)];
        eval_targets<R>(J, i, ws, f0, qx, qy, t < total && j != i, o_fl, j, lane, item, slots, fx, fy, en);
    }
}

// Inclusive prefix sum of x over the warp.
__device__ __forceinline__ int warp_incl_scan(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(CSS_FULL, x, o);
        if (lane >= o) x += t;
    }
    return x;
}

// The lane whose inclusive-scan range holds item t (31 for t beyond the total).
__device__ __forceinline__ int scan_owner(int incl, int t) {
    int owner = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int v = __shfl_sync(CSS_FULL, incl, owner + step - 1);
        if (v <= t) owner += step;
    }
    return min(owner, 31);
}

// Per-warp staging (shared memory) of a wave's vertex candidates and then of its children,
// so that each round takes 32 of them whatever lane produced them; the two phases use the
// union in turn, and after the waves it holds the source's targets.  The children held over
// from one wave to the next sit beside it.
template <class R>
struct WaveStage {
    union {
        VCand<R, false> vc[3][32];
        Win<R> ch[2][32];
        int2 tq[2 * 32 * sizeof(Win<R>) / sizeof(int2)];   // (face, particle) targets, after the waves
    };
    Win<R> carry[CARRY_CAP];
};

template <class R, int SH>
__device__ void run_source(const cssi::GeoJob& J, int i, Ws<R, SH>& ws, WarpSm& sm, WaveStage<R>* stg, int lane,
                           int* status, unsigned long long* counters, int item, int32_t* defer_list,
                           int* defer_count) {
    const DMesh& m = J.m;
    const double rc = J.rc;
    const int f0 = J.face[i];
    const double* b = J.bary + 3 * (size_t)i;
    const double qxd = b[1] * m.lay[3 * f0] + b[2] * m.lay[3 * f0 + 1];
    const double qyd = b[2] * m.lay[3 * f0 + 2];
    seed_source<R>(m, ws, sm, f0, qxd, qyd, rc, lane);
    unsigned long long n_prop = 0;
    const int max_waves = 4 * ws.wcap + 64;
    for (int wave = 0;; ++wave) {
        __syncwarp();
        const int npend = min(sm.npend, ws.wcap);
        const int ncar = SH == 2 ? 0 : sm.ncar;
        if ((npend == 0 && sm.nemit == 0 && ncar == 0) || sm.err) break;
        if (wave > max_waves) { if (lane == 0) atomicOr(&sm.err, css::ST_ITER_LIMIT); break; }
        float kmin, kmax;
        pending_range<R>(ws, npend, lane, kmin, kmax);
        // vertices whose distance no queued or held-over window can improve emit first (none
        // can while the smallest queued distance bound exceeds the smallest key).  Their
        // windows join the held-over ones, for this wave's insertion rounds, as far as there is
        // room; the rest go in at once, and once the queue has changed its smallest keys are
        // looked at again
        float kemit = npend ? kmin : INFINITY;
        if (ncar) kemit = fminf(kemit, __uint_as_float(sm.cmin));
        int ncar2 = ncar;
        if constexpr (SH != 2) {
            if (sm.nemit > 0 && ((!npend && !ncar) || __uint_as_float(sm.emin) <= kemit)) {
                const int npraw = sm.npend;
                emit_round<R>(m, ws, sm, rc, (double)kemit, lane, stg->carry + ncar, CARRY_CAP - ncar, &sm.nstg);
                __syncwarp();
                const int ns = sm.nstg;
                if (ns > 0) {
                    const float kk = lane < ns ? __double2float_rd((double)win_key<R>(stg->carry[ncar + lane])) : INFINITY;
                    const float km = __uint_as_float(__reduce_min_sync(CSS_FULL, __float_as_uint(kk)));
                    __syncwarp();
                    if (lane == 0) { sm.ncar = ncar + ns; sm.cmin = min(sm.cmin, __float_as_uint(km)); }
                    __syncwarp();
                    ncar2 = ncar + ns;
                }
                if (sm.npend != npraw) continue;
            }
        } else {
            if (sm.nemit > 0 && ((!npend && !ncar) || __uint_as_float(sm.emin) <= kemit) &&
                emit_round<R>(m, ws, sm, rc, (double)kemit, lane) > 0)
                continue;
        }
        if (npend == 0 && ncar2 == 0) continue;
        // with nothing queued the held-over windows go in now, whatever their edges
        const int idx = npend ? select_wave<R>(ws, sm, npend, kmin, kmax, lane) : -1;
        Win<R> w;
        bool act = false;
        if (idx >= 0) {
            w = ws.win[idx];
            act = (w.flags & WIN_ALIVE) && !(w.flags & WIN_DONE) && (double)win_key<R>(w) < rc;
            if (act) ws.win[idx].flags = w.flags | WIN_DONE;
        }
        VCand<R, SH == 2> vc[3];
        Win<R> ch[2];
        int nvc = 0, nch = 0;
        if (act) propagate<R, SH == 2>(m, w, rc, vc, nvc, ch, nch);
        n_prop += __popc(__ballot_sync(CSS_FULL, act));
        __syncwarp();
        // one call site per round kind keeps the kernel's instruction footprint small
        // (divergent insertion code otherwise thrashes the instruction cache)
        if constexpr (SH == 2) {   // the path kernel: one round per candidate slot
#pragma unroll 1
            for (int q = 0; q < 3; ++q)
                vertex_round<R>(m, ws, sm, q < nvc, q == 0 ? vc[0] : (q == 1 ? vc[1] : vc[2]), rc, lane);
#pragma unroll 1
            for (int q = 0; q < 2; ++q) child_round<R>(m, ws, sm, q < nch, q == 0 ? ch[0] : ch[1], rc, lane);
        } else {
            // the wave's vertex candidates (up to three a lane), 32 to a round
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (q < nvc) stg->vc[q][lane] = vc[q];
            __syncwarp();
            const int vi = warp_incl_scan(nvc, lane);
            const int vt = __shfl_sync(CSS_FULL, vi, 31);
#pragma unroll 1
            for (int base = 0; base < vt; base += 32) {
                const int t = base + lane;
                const int owner = scan_owner(vi, t);
                const int slot = t - (__shfl_sync(CSS_FULL, vi, owner) - __shfl_sync(CSS_FULL, nvc, owner));
                VCand<R, false> c;
                const bool has = t < vt;
                if (has) c = stg->vc[slot][owner];
                vertex_round<R>(m, ws, sm, has, c, rc, lane);
            }
            __syncwarp();
            // then the children held over from the last wave and its own (up to two a lane), 32
            // to a round; the held-over ones all fall in the first round
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (q < nch) stg->ch[q][lane] = ch[q];
            __syncwarp();
            const int ci = warp_incl_scan(nch, lane);
            const int ct = __shfl_sync(CSS_FULL, ci, 31) + ncar2;
#pragma unroll 1
            for (int base = 0; base < ct; base += 32) {
                const int t = base + lane;
                const int owner = scan_owner(ci, t - ncar2);
                const int slot = t - ncar2 - (__shfl_sync(CSS_FULL, ci, owner) - __shfl_sync(CSS_FULL, nch, owner));
                Win<R> c;
                const bool has = t < ct;
                if (t < ncar2) c = stg->carry[t];
                else if (has) c = stg->ch[slot][owner];
                if (base == 0 && ncar2) {
                    __syncwarp();
                    if (lane == 0) { sm.ncar = 0; sm.cmin = 0x7f800000u; }
                    __syncwarp();
                }
                child_round<R>(m, ws, sm, has, c, rc, lane, npend ? stg->carry : nullptr, &sm.ncar);
            }
            __syncwarp();
        }
    }
    __syncwarp();
    const int err = sm.err;
    // a patch too large for this pass's tables or pool: hand the source to the second pass
    if (defer_list && (err & (css::ST_WIN_OVERFLOW | css::ST_HASH_OVERFLOW | css::ST_ITER_LIMIT))) {
        if (lane == 0) {
            defer_list[atomicAdd(defer_count, 1)] = item;
            atomicAdd(counters + 4, 1ull);
        }
        __syncwarp();
        return;
    }
    const int nface = min(sm.nface, ws.fcap);
    // ---- target evaluation (+ forces)
    const R qx = (R)qxd, qy = (R)qyd;
    double fx = 0.0, fy = 0.0, en = 0.0;
    int npair = 0;
    const bool wp = J.want_pairs != 0;
    auto slots = [&](unsigned pm) { const int b = npair; npair += __popc(pm); return b; };
    if constexpr (SH == 2) {
        for (int fb = 0; fb < nface; fb += 32)
            eval_face_block<R>(J, i, ws, f0, qx, qy, fb, nface, lane, item, slots, fx, fy, en);
    } else {
        // the targets of all the faces are gathered in the stage first and then evaluated 32 at a
        // time (a block of 32 faces holds only a few particles on the sparse workloads)
        constexpr int TQ = (int)(sizeof(WaveStage<R>::tq) / sizeof(int2));
        int2* tq = stg->tq;
        int nt = 0;
        // one loop, one evaluation site (instruction footprint): each turn either reads the
        // next block of 32 faces, queues up to 32 of its targets, or evaluates the queue (when
        // it could not take another 32, or at the end)
        int fb = 0, tb = 0, total = 0, incl = 0, fl = -1, st = 0, cnt = 0;
#pragma unroll 1
        for (;;) {
            if (fb < nface && tb >= total) {   // the next block's buckets
                const int fi = fb + lane;
                fl = -1; st = 0; cnt = 0;
                if (fi < nface) {
                    fl = ws.flist[fi];
                    const int key = m.frank ? m.frank[fl] : fl;
                    st = J.fstart[key];
                    cnt = J.fstart[key + 1] - st;
                }
                incl = warp_incl_scan(cnt, lane);
                total = __shfl_sync(CSS_FULL, incl, 31);
                tb = 0;
                if (total == 0) { fb += 32; continue; }
            }
            const bool done = fb >= nface;
            if (done || nt + 32 > TQ) {
                __syncwarp();
#pragma unroll 1
                for (int base = 0; base < nt; base += 32) {
                    const bool has = base + lane < nt;
                    const int2 e = has ? tq[base + lane] : make_int2(-1, -1);
                    eval_targets<R>(J, i, ws, f0, qx, qy, has, e.x, e.y, lane, item, slots, fx, fy, en);
                }
                __syncwarp();
                nt = 0;
                if (done) break;
                continue;
            }
            const int t = tb + lane;
            const int owner = scan_owner(incl, t);
            const int o_fl = __shfl_sync(CSS_FULL, fl, owner);
            const int o_st = __shfl_sync(CSS_FULL, st, owner);
            const int o_ex = __shfl_sync(CSS_FULL, incl - cnt, owner);
            int j = -1;
            if (t < total) j = J.fitems[o_st + (t - o_ex)];
            const bool valid = t < total && j != i;
            const unsigned vm = __ballot_sync(CSS_FULL, valid);
            if (valid) tq[nt + __popc(vm & css::lanemask_lt())] = make_int2(o_fl, j);
            nt += __popc(vm);
            tb += 32;
            if (tb >= total) fb += 32;
        }
    }
    fx = css::warp_sum(fx);
    fy = css::warp_sum(fy);
    en = css::warp_sum(en);
    if (lane == 0) {
        if (J.want_forces) {
            const double* fr = m.frame + 9 * (size_t)f0;
            J.force[3 * (size_t)i] = fx * fr[3] + fy * fr[6];
            J.force[3 * (size_t)i + 1] = fx * fr[4] + fy * fr[7];
            J.force[3 * (size_t)i + 2] = fx * fr[5] + fy * fr[8];
            if (J.epot) atomicAdd(J.epot, en);
        }
        if (J.pcnt) J.pcnt[i] = npair;
        int st = err;
        if (wp && npair > J.pair_cap) st |= css::ST_PAIR_OVERFLOW;
        if (st) atomicOr(status, st);
        atomicAdd(counters + 0, 1ull);
        atomicAdd(counters + 1, (unsigned long long)min(sm.nwin, ws.wcap));
        atomicAdd(counters + 2, n_prop);
        atomicAdd(counters + 3, (unsigned long long)npair);
    }
    __syncwarp();
}

// ------------------------------------------------------------------ team form
// The W warps of a CTA work on one source.  For sets with fewer sources than resident warps
// one warp per source leaves SMs idle and the launch lasts one source's chain; a team makes
// each wave W times wider and spreads the insertions over W warps.  Every wave warp 0 picks
// up to 32 W pending windows; each warp unfolds 32 of them; the children and vertex
// candidates are staged in shared memory in (warp, lane, slot) order, and warp w inserts
// those whose edge (vertex) id is w modulo W, so no two warps ever touch one edge list or
// one vertex entry (the hash tables, the pool and the queues take concurrent claims through
// atomics); emissions run on warp 0 between waves while the others wait.  Barriers separate
// the phases, and every loop containing one has a trip count that is the same for all
// threads of the CTA (read from shared memory after a barrier).
constexpr int MAX_TEAM = 8;

struct TeamSm {
    int item;         // the team's current work item (>= nitems: none left)
    int action;       // next step of the wave loop: 0 finished, 1 look again, 2 unfold nsel windows
                      // (and insert the staged emitted windows with their children), 3 insert
                      // the staged emitted windows and the held-over ones
    int nsel;
    int nstaged;      // emitted windows staged (in their own area) for the whole team to insert
    int npair;        // slots taken in the source's pair row
    int ncar[MAX_TEAM];   // windows each warp holds over to the next wave
    double fx[MAX_TEAM], fy[MAX_TEAM], en[MAX_TEAM];
    unsigned long long nprop[MAX_TEAM];
    int sel[32 * MAX_TEAM];
};

// shared memory of a team besides the static part: its tables (shared placement), then the
// staged children (64 per warp), vertex candidates (96 per warp), the warps' owned-index
// lists, their held-over windows (32 per warp) and the staged emitted windows (32 per warp)
template <class R>
__host__ __device__ inline size_t team_child_off(int shared_scale) {
    return al16(shared_scale ? sh_bytes_per_warp<R>(shared_scale) : 0);
}
template <class R>
__host__ __device__ inline size_t team_vcand_off(int shared_scale, int W) {
    return team_child_off<R>(shared_scale) + al16((size_t)64 * W * sizeof(Win<R>));
}
template <class R>
__host__ __device__ inline size_t team_idx_off(int shared_scale, int W) {
    return team_vcand_off<R>(shared_scale, W) + al16((size_t)96 * W * sizeof(VCand<R, false>));
}
template <class R>
__host__ __device__ inline size_t team_car_off(int shared_scale, int W) {
    return team_idx_off<R>(shared_scale, W) + al16((size_t)96 * W * W * sizeof(int));
}
template <class R>
__host__ __device__ inline size_t team_emit_off(int shared_scale, int W) {
    return team_car_off<R>(shared_scale, W) + al16((size_t)CARRY_CAP * W * sizeof(Win<R>));
}
template <class R>
__host__ __device__ inline size_t team_smem_bytes(int shared_scale, int W) {
    return team_emit_off<R>(shared_scale, W) + (size_t)32 * W * sizeof(Win<R>);
}

// The next wave of a team: as select_wave, with up to `cap` windows written to sel[]
// (run by one warp); returns how many were taken.
template <class R, int SH>
__device__ int select_wave_cap(Ws<R, SH>& ws, WarpSm& sm, int npend, float kmin, float kmax, int lane, int cap,
                               int* sel) {
    float T = kmax;
    if (npend > cap) {
        float lo = kmin, hi = kmax;
        for (int it = 0; it < 12; ++it) {
            const float mid = 0.5f * (lo + hi);
            if (!(mid > lo && mid < hi)) break;
            int c = 0;
            for (int i = lane; i < npend; i += 32) c += ws.pk[i] <= mid ? 1 : 0;
            c = (int)__reduce_add_sync(CSS_FULL, (unsigned)c);
            if (c < cap) lo = mid;
            else {
                hi = mid;
                T = mid;
                if (c <= 2 * cap) break;
            }
        }
    }
    int taken = 0, kept = 0;
    for (int base = 0; base < npend; base += 32) {
        const int i = base + lane;
        int id = -1;
        float k = 0.0f;
        if (i < npend) { id = ws.pq[i]; k = ws.pk[i]; }
        __syncwarp();
        const bool cand = i < npend && k <= T;
        const unsigned cm = __ballot_sync(CSS_FULL, cand);
        const int r = taken + __popc(cm & css::lanemask_lt());
        const bool take = cand && r < cap;
        const bool keep = i < npend && !take;
        const unsigned km = __ballot_sync(CSS_FULL, keep);
        if (take) sel[r] = id;
        if (keep) {   // kept entries move forward only: p <= i
            const int p = kept + __popc(km & css::lanemask_lt());
            ws.pq[p] = id;
            ws.pk[p] = k;
        }
        taken = min(cap, taken + __popc(cm));
        kept += __popc(km);
    }
    __syncwarp();
    if (lane == 0) sm.npend = kept;
    __syncwarp();
    return taken;
}

// One source processed by the team of the W warps of this CTA (see the team form above).
// The staged windows cst[0 .. count) (he < 0: an empty slot) inserted by the team: each warp
// lists those on the edges it owns (undirected edge id modulo W), in order, and inserts them
// 32 to a round.
template <class R, int SH>
__device__ __forceinline__ void team_insert(const DMesh& m, Ws<R, SH>& ws, WarpSm& sm, const Win<R>* cst, int count,
                                            const Win<R>* est, int count2, int* ilist, int W, int wid, int lane,
                                            double rc, Win<R>* wcar, int* ncar, bool hold) {
    // staged entry s: the children cst[0, count), then the emitted windows est[0, count2)
    int nown = 0;
    const int all = count + count2;
    for (int base = 0; base < all; base += 32) {
        const int s = base + lane;
        bool own = false;
        if (s < all) {
            const int he = s < count ? cst[s].he : est[s - count].he;
            own = he >= 0 && m.edge[he] % W == wid;
        }
        const unsigned om = __ballot_sync(CSS_FULL, own);
        if (own) ilist[nown + __popc(om & css::lanemask_lt())] = s;
        nown += __popc(om);
    }
    __syncwarp();
    // the windows this warp held over (all of them in the first round), then the staged ones
    // on its edges; with hold, same-edge windows after the first wait for the next wave
    const int nc = *ncar;
    const int total = nc + nown;
    for (int base = 0; base < total; base += 32) {
        const int t = base + lane;
        Win<R> c;
        const bool has = t < total;
        if (t < nc) c = wcar[t];
        else if (has) {
            const int s = ilist[t - nc];
            c = s < count ? cst[s] : est[s - count];
        }
        if (base == 0 && nc) {
            __syncwarp();
            if (lane == 0) *ncar = 0;
            __syncwarp();
        }
        child_round<R>(m, ws, sm, has, c, rc, lane, hold ? wcar : nullptr, ncar);
    }
}

template <class R, int SH>
__device__ void run_source_team(const cssi::GeoJob& J, int i, Ws<R, SH>& ws, WarpSm& sm, TeamSm& tm, Win<R>* cst,
                                VCand<R, false>* vst, int* ilist, Win<R>* wcar, Win<R>* est, int W, int wid, int lane,
                                int* status,
                                unsigned long long* counters, int item, int32_t* defer_list, int* defer_count) {
    const DMesh& m = J.m;
    const double rc = J.rc;
    const int f0 = J.face[i];
    const double* b = J.bary + 3 * (size_t)i;
    const double qxd = b[1] * m.lay[3 * f0] + b[2] * m.lay[3 * f0 + 1];
    const double qyd = b[2] * m.lay[3 * f0 + 2];
    if (wid == 0) {
        seed_source<R>(m, ws, sm, f0, qxd, qyd, rc, lane);
        if (lane == 0) tm.npair = 0;
    }
    if (lane == 0) tm.ncar[wid] = 0;
    __syncthreads();
    unsigned long long n_prop = 0;
    const int max_waves = 4 * ws.wcap + 64;
    for (int wave = 0;; ++wave) {
        // warp 0: emissions and the wave's selection; the others wait at the barrier
        if (wid == 0) {
            __syncwarp();
            int act = 2;
            const int npend = min(sm.npend, ws.wcap);
            int ncar = 0;   // windows the warps hold over
            for (int w2 = 0; w2 < W; ++w2) ncar += tm.ncar[w2];
            if ((npend == 0 && sm.nemit == 0 && ncar == 0) || sm.err) act = 0;
            else if (wave > max_waves) {
                if (lane == 0) atomicOr(&sm.err, css::ST_ITER_LIMIT);
                act = 0;
            } else {
                float kmin, kmax;
                pending_range<R>(ws, npend, lane, kmin, kmax);
                float kemit = npend ? kmin : INFINITY;   // held-over windows bound it too
                if (ncar) kemit = fminf(kemit, __uint_as_float(sm.cmin));
                // the emitted windows are staged for this step's insertion; those that do not
                // fit go in at once, and once the queue has changed its smallest keys are
                // looked at again
                int nst = 0;
                bool again = false;
                if (sm.nemit > 0 && ((!npend && !ncar) || __uint_as_float(sm.emin) <= kemit)) {
                    const int npraw = sm.npend;
                    emit_round<R>(m, ws, sm, rc, (double)kemit, lane, est, 32 * W, &tm.nstaged);
                    __syncwarp();
                    nst = tm.nstaged;
                    again = sm.npend != npraw;
                } else if (lane == 0) tm.nstaged = 0;
                if (again) act = nst > 0 ? 3 : 1;
                else if (npend == 0) act = (ncar || nst) ? 3 : 1;   // nothing queued: they go in now
                else {
                    const int taken = select_wave_cap<R>(ws, sm, npend, kmin, kmax, lane, 32 * W, tm.sel);
                    if (lane == 0) tm.nsel = taken;
                }
            }
            __syncwarp();
            if (lane == 0) {
                tm.action = act;
                // every held-over window is taken up by this step's insertion; those held over
                // again set the bound anew
                if (act >= 2 && ncar) sm.cmin = 0x7f800000u;
            }
        }
        __syncthreads();
        const int act = tm.action;
        const int nsel = tm.nsel;
        const int nstaged = tm.nstaged;
        __syncthreads();   // everyone has read the decision before warp 0 writes the next one
        if (act == 0) break;
        if (act == 1) continue;
        if (act == 3) {   // the emitted windows warp 0 staged, inserted by their edges' owners
            team_insert<R>(m, ws, sm, cst, 0, est, nstaged, ilist, W, wid, lane, rc, wcar, &tm.ncar[wid], false);
            __syncthreads();
            continue;
        }
        // every warp unfolds its 32 windows and stages what they produce
        const int k = wid * 32 + lane;
        Win<R> w;
        bool on = false;
        if (k < nsel) {
            const int idx = tm.sel[k];
            w = ws.win[idx];
            on = (w.flags & WIN_ALIVE) && !(w.flags & WIN_DONE) && (double)win_key<R>(w) < rc;
            if (on) ws.win[idx].flags = w.flags | WIN_DONE;
        }
        VCand<R, false> vc[3];
        Win<R> ch[2];
        int nvc = 0, nch = 0;
        if (on) propagate<R, false>(m, w, rc, vc, nvc, ch, nch);
        n_prop += __popc(__ballot_sync(CSS_FULL, on));
#pragma unroll 1
        for (int q = 0; q < 3; ++q) {
            VCand<R, false> c = q == 0 ? vc[0] : (q == 1 ? vc[1] : vc[2]);
            if (q >= nvc) c.v = -1;
            vst[3 * k + q] = c;
        }
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            Win<R> c = q == 0 ? ch[0] : ch[1];
            if (q >= nch) c.he = -1;
            cst[2 * k + q] = c;
        }
        __syncthreads();
        // each warp lists the staged vertex candidates it owns (vertex id modulo W), in order,
        // and takes them 32 to a round
        int nown = 0;
        for (int base = 0; base < 3 * nsel; base += 32) {
            const int s = base + lane;
            const bool own = s < 3 * nsel && vst[s].v >= 0 && vst[s].v % W == wid;
            const unsigned om = __ballot_sync(CSS_FULL, own);
            if (own) ilist[nown + __popc(om & css::lanemask_lt())] = s;
            nown += __popc(om);
        }
        __syncwarp();
        for (int base = 0; base < nown; base += 32) {
            VCand<R, false> c;
            const bool has = base + lane < nown;
            if (has) c = vst[ilist[base + lane]];
            vertex_round<R>(m, ws, sm, has, c, rc, lane);
        }
        __syncthreads();
        // and the staged children on the edges it owns (undirected edge id modulo W)
        team_insert<R>(m, ws, sm, cst, 2 * nsel, est, nstaged, ilist, W, wid, lane, rc, wcar, &tm.ncar[wid], true);
        __syncthreads();
    }
    const int err = sm.err;
    // a patch too large for this pass's tables or pool: hand the source to the second pass
    if (defer_list && (err & (css::ST_WIN_OVERFLOW | css::ST_HASH_OVERFLOW | css::ST_ITER_LIMIT))) {
        if (wid == 0 && lane == 0) {
            defer_list[atomicAdd(defer_count, 1)] = item;
            atomicAdd(counters + 4, 1ull);
        }
        return;
    }
    // target evaluation: warp w takes the face blocks w, w + W, ...; pair slots from the
    // team's counter; forces summed per warp, then over the warps in order
    const int nface = min(sm.nface, ws.fcap);
    const R qx = (R)qxd, qy = (R)qyd;
    double fx = 0.0, fy = 0.0, en = 0.0;
    for (int fb = 32 * wid; fb < nface; fb += 32 * W)
        eval_face_block<R>(J, i, ws, f0, qx, qy, fb, nface, lane, item,
                           [&](unsigned pm) {
                               int base = 0;
                               if (lane == 0 && pm) base = atomicAdd(&tm.npair, __popc(pm));
                               return __shfl_sync(CSS_FULL, base, 0);
                           },
                           fx, fy, en);
    fx = css::warp_sum(fx);
    fy = css::warp_sum(fy);
    en = css::warp_sum(en);
    if (lane == 0) {
        tm.fx[wid] = fx;
        tm.fy[wid] = fy;
        tm.en[wid] = en;
        tm.nprop[wid] = n_prop;
    }
    __syncthreads();
    if (wid == 0 && lane == 0) {
        double sx = 0.0, sy = 0.0, se = 0.0;
        unsigned long long np = 0;
        for (int w2 = 0; w2 < W; ++w2) {
            sx += tm.fx[w2];
            sy += tm.fy[w2];
            se += tm.en[w2];
            np += tm.nprop[w2];
        }
        const int npair = tm.npair;
        if (J.want_forces) {
            const double* fr = m.frame + 9 * (size_t)f0;
            J.force[3 * (size_t)i] = sx * fr[3] + sy * fr[6];
            J.force[3 * (size_t)i + 1] = sx * fr[4] + sy * fr[7];
            J.force[3 * (size_t)i + 2] = sx * fr[5] + sy * fr[8];
            if (J.epot) atomicAdd(J.epot, se);
        }
        if (J.pcnt) J.pcnt[i] = npair;
        int st = err;
        if (J.want_pairs && npair > J.pair_cap) st |= css::ST_PAIR_OVERFLOW;
        if (st) atomicOr(status, st);
        atomicAdd(counters + 0, 1ull);
        atomicAdd(counters + 1, (unsigned long long)min(sm.nwin, ws.wcap));
        atomicAdd(counters + 2, np);
        atomicAdd(counters + 3, (unsigned long long)npair);
    }
}

// Team kernel: one CTA (W = blockDim / 32 warps, 2..8) per source at a time, persistent over
// the work items; one workspace slice per CTA (g.nwarps counts teams).
template <class R, int OCC, int SH>
__global__ void __launch_bounds__(256, OCC) k_geodesic_team(const __grid_constant__ cssi::GeoJob job0,
                                                       const cssi::GeoJob* jobs, cssi::GeoQueue q, cssi::GeoWs g,
                                                       int* work, int* status, unsigned long long* counters) {
    static_assert(SH != 2, "the path form runs one warp per source");
    __shared__ WarpSm sm;
    __shared__ TeamSm tm;
    __shared__ Ws<R, SH> ws;
    const int W = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int team = blockIdx.x;
    if (team >= g.nwarps) return;   // the whole CTA
    extern __shared__ __align__(16) unsigned char dsm[];
    Win<R>* cst = (Win<R>*)(dsm + team_child_off<R>(g.shared));
    VCand<R, false>* vst = (VCand<R, false>*)(dsm + team_vcand_off<R>(g.shared, W));
    int* ilist = (int*)(dsm + team_idx_off<R>(g.shared, W)) + (size_t)wid * 96 * W;   // this warp's list
    Win<R>* wcar = (Win<R>*)(dsm + team_car_off<R>(g.shared, W)) + (size_t)wid * CARRY_CAP;
    Win<R>* est = (Win<R>*)(dsm + team_emit_off<R>(g.shared, W));
    uint32_t gen = 0;
    if (threadIdx.x == 0) {
        ws = ws_bind<R, SH>(g, team);
        if constexpr (SH == 1) ws_bind_shared<R, SH>(ws, dsm, g.shared);
        gen = g.gen[team];
    }
    __syncthreads();
    const int nitems = q.item_count ? min(*(volatile const int*)q.item_count, q.nitems) : q.nitems;
    for (;;) {
        if (threadIdx.x == 0) tm.item = atomicAdd(work, 1);
        __syncthreads();
        const int k = tm.item;
        if (k >= nitems) break;
        const int item = q.item_list ? q.item_list[k] : k;
        const int jid = q.job_of_item ? q.job_of_item[item] : 0;
        const cssi::GeoJob& J = jobs ? jobs[jid] : job0;
        const int pos = q.src_of_item ? q.src_of_item[item] : item;
        const int src = J.order ? J.order[pos] : pos;
        if (threadIdx.x == 0) {
            ++gen;
            if (gen == 0) gen = 1;   // 0 marks never-used entries
            ws.gen = gen;
        }
        __syncthreads();
        run_source_team<R>(J, src, ws, sm, tm, cst, vst, ilist, wcar, est, W, wid, lane, status, counters, item,
                           q.defer_list, q.defer_count);
        __syncthreads();   // the team's state is free before the next claim
    }
    if (threadIdx.x == 0) g.gen[team] = gen;
}

// OCC = CTAs of 256 threads per SM the register budget must allow: 1 gives up to 255
// registers a thread (fewer resident warps, no spills), 2 caps them at 128 (twice the
// resident warps, some spills); which is faster depends on the workload.
// The warp's workspace descriptor (warp-uniform pointers and sizes) lives in shared memory:
// the out-of-line rounds take it by reference, and a descriptor in registers would be
// copied to each thread's local memory for that.  The job parameter is a grid constant for
// the same reason (its address is taken without a local copy).
template <class R, int OCC, int SH>
__global__ void __launch_bounds__(256, OCC) k_geodesic(const __grid_constant__ cssi::GeoJob job0, const cssi::GeoJob* jobs,
                                                  cssi::GeoQueue q, cssi::GeoWs g, int* work, int* status,
                                                  unsigned long long* counters) {
    __shared__ WarpSm smem[MAX_WARPS_CTA];
    __shared__ Ws<R, SH> wsm[MAX_WARPS_CTA];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    if (gw >= g.nwarps) return;
    WarpSm& sm = smem[wib];
    Ws<R, SH>& ws = wsm[wib];
    extern __shared__ __align__(16) unsigned char dsm[];
    if (lane == 0) {
        ws = ws_bind<R, SH>(g, gw);
        if constexpr (SH == 1) ws_bind_shared<R, SH>(ws, dsm + (size_t)wib * sh_bytes_per_warp<R>(g.shared), g.shared);
    }
    // the wave staging buffers follow the CTA's tables
    WaveStage<R>* stg = nullptr;
    if constexpr (SH != 2)
        stg = reinterpret_cast<WaveStage<R>*>(
                  dsm + (SH == 1 ? (size_t)(blockDim.x >> 5) * sh_bytes_per_warp<R>(g.shared) : 0)) + wib;
    __syncwarp();
    uint32_t gen = 0;
    if (lane == 0) gen = g.gen[gw];
    gen = __shfl_sync(CSS_FULL, gen, 0);
    // the second pass takes its work items from the first pass's deferral list
    const int nitems = q.item_count ? min(*(volatile const int*)q.item_count, q.nitems) : q.nitems;
    const int tile = max(1, q.tile);
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(work, tile);
        base = __shfl_sync(CSS_FULL, base, 0);
        if (base >= nitems) break;
        const int end = min(base + tile, nitems);
        for (int k = base; k < end; ++k) {
            const int item = q.item_list ? q.item_list[k] : k;
            const int jid = q.job_of_item ? q.job_of_item[item] : 0;
            const cssi::GeoJob& J = jobs ? jobs[jid] : job0;
            const int pos = q.src_of_item ? q.src_of_item[item] : item;   // position in the set's order
            const int src = J.order ? J.order[pos] : pos;
            ++gen;
            if (gen == 0) gen = 1;   // 0 marks never-used entries
            __syncwarp();
            if (lane == 0) ws.gen = gen;
            __syncwarp();
            run_source<R>(J, src, ws, sm, stg, lane, status, counters, item, q.defer_list, q.defer_count);
        }
    }
    if (lane == 0) g.gen[gw] = gen;
}

// CSR compaction: rows sorted by neighbour index
__global__ void k_compact(int32_t n, const int32_t* pcnt, const int32_t* pj, const double* pd, const double* pt,
                          int pair_cap, const int64_t* row_start, int32_t* oj, double* od, double* ot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = min(pcnt[i], pair_cap);
    const int64_t o = row_start[i];
    const size_t s = (size_t)i * pair_cap;
    for (int a = 0; a < c; ++a) { oj[o + a] = pj[s + a]; od[o + a] = pd[s + a];
        ot[3 * (o + a)] = pt[3 * (s + a)]; ot[3 * (o + a) + 1] = pt[3 * (s + a) + 1]; ot[3 * (o + a) + 2] = pt[3 * (s + a) + 2]; }
    for (int a = 1; a < c; ++a) {           // insertion sort by j (rows are short)
        const int32_t kj = oj[o + a];
        const double kd = od[o + a], k0 = ot[3 * (o + a)], k1 = ot[3 * (o + a) + 1], k2 = ot[3 * (o + a) + 2];
        int b = a - 1;
        while (b >= 0 && oj[o + b] > kj) {
            oj[o + b + 1] = oj[o + b]; od[o + b + 1] = od[o + b];
            ot[3 * (o + b + 1)] = ot[3 * (o + b)]; ot[3 * (o + b + 1) + 1] = ot[3 * (o + b) + 1]; ot[3 * (o + b + 1) + 2] = ot[3 * (o + b) + 2];
            --b;
        }
        oj[o + b + 1] = kj; od[o + b + 1] = kd; ot[3 * (o + b + 1)] = k0; ot[3 * (o + b + 1) + 1] = k1; ot[3 * (o + b + 1) + 2] = k2;
    }
}

}  // namespace

namespace cssi {

size_t geo_ws_bytes_per_warp(int precision, int win_cap, int tab_cap, int* log_eh, int* log_vh, int* log_fh,
                             int* fcap, int* emcap) {
    // hash tables sized from tab_cap (0: from the window capacity): tab_cap edge slots, half
    // as many vertex slots, tab_cap face slots (a patch of tab_cap / 2 faces at load 1/2).
    // Tables much larger than the patches a pass sees spread each source's entries over
    // many cache lines; a source that overflows them is deferred like one that overflows
    // the pool.
    const int t = tab_cap > 0 ? tab_cap : win_cap;
    int le = 6, lv = 6, lf = 6;
    while ((1 << le) < t) ++le;
    while ((1 << lv) < t / 2) ++lv;
    while ((1 << lf) < t) ++lf;
    *log_eh = le; *log_vh = lv; *log_fh = lf;
    *fcap = 1 << (lf - 1);
    *emcap = 1 << lv;
    size_t off[13];
    return precision == CSS_FP32 ? ws_layout<float>(le, lv, lf, win_cap, *fcap, *emcap, off)
                                 : ws_layout<double>(le, lv, lf, win_cap, *fcap, *emcap, off);
}

size_t geodesic_shared_bytes(int precision, int warps_per_cta, int shared_scale) {
    const bool f32 = precision == CSS_FP32;
    const size_t stage = f32 ? sizeof(WaveStage<float>) : sizeof(WaveStage<double>);
    const size_t tables = !shared_scale ? 0 : (f32 ? sh_bytes_per_warp<float>(shared_scale)
                                                   : sh_bytes_per_warp<double>(shared_scale));
    return (size_t)warps_per_cta * (tables + stage);
}

cudaError_t launch_geodesic(const GeoJob& job0, const GeoJob* djobs, const GeoQueue& q, int precision,
                            const GeoWs& ws, int warps_per_cta, int nctas, int* work_counter, int* status,
                            unsigned long long* counters, cudaStream_t st) {
    const dim3 block(32 * warps_per_cta);
    const size_t sm = geodesic_shared_bytes(precision, warps_per_cta, ws.shared);
    // one instantiation per (precision, register budget, table placement)
    const bool light = ws.occupancy == 2, sh = ws.shared != 0;
#define CSS_LAUNCH(RT, O, S) k_geodesic<RT, O, S><<<nctas, block, sm, st>>>(job0, djobs, q, ws, work_counter, status, counters)
    if (precision == CSS_FP32) {
        if (light) { if (sh) CSS_LAUNCH(float, 2, true); else CSS_LAUNCH(float, 2, false); }
        else { if (sh) CSS_LAUNCH(float, 1, true); else CSS_LAUNCH(float, 1, false); }
    } else {
        if (light) { if (sh) CSS_LAUNCH(double, 2, true); else CSS_LAUNCH(double, 2, false); }
        else { if (sh) CSS_LAUNCH(double, 1, true); else CSS_LAUNCH(double, 1, false); }
    }
#undef CSS_LAUNCH
    return cudaGetLastError();
}

size_t geo_link_bytes_per_warp(int log_vh) {
    const size_t VH = (size_t)1 << log_vh;
    return 2 * al16(VH * 4) + al16(VH * 24);
}

cudaError_t launch_geodesic_links(const GeoJob& job, const GeoQueue& q, const GeoWs& ws, int warps_per_cta,
                                  int nctas, int* work_counter, int* status, unsigned long long* counters,
                                  cudaStream_t st) {
    k_geodesic<double, 1, 2><<<nctas, 32 * warps_per_cta, 0, st>>>(job, nullptr, q, ws, work_counter, status, counters);
    return cudaGetLastError();
}

// resident CTAs per SM for a launch shape (0: the shape does not fit an SM)
template <class R, int OCC, int SH>
static int blocks_per_sm(int warps_per_cta, size_t dyn) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_geodesic<R, OCC, SH>) != cudaSuccess) { cudaGetLastError(); return 0; }
    const int room = optin - (int)fa.sharedSizeBytes;   // dynamic shared memory a CTA may take
    if (dyn > (size_t)room) return 0;
    if (cudaFuncSetAttribute(k_geodesic<R, OCC, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, room) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_geodesic<R, OCC, SH>, 32 * warps_per_cta, dyn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

int geodesic_blocks_per_sm(int precision, int warps_per_cta, int shared_scale, int occupancy) {
    const size_t dyn = geodesic_shared_bytes(precision, warps_per_cta, shared_scale);
    const bool f32 = precision == CSS_FP32, sh = shared_scale != 0;
    if (occupancy == 2) {
        if (sh) return f32 ? blocks_per_sm<float, 2, true>(warps_per_cta, dyn) : blocks_per_sm<double, 2, true>(warps_per_cta, dyn);
        return f32 ? blocks_per_sm<float, 2, false>(warps_per_cta, dyn) : blocks_per_sm<double, 2, false>(warps_per_cta, dyn);
    }
    if (sh) return f32 ? blocks_per_sm<float, 1, true>(warps_per_cta, dyn) : blocks_per_sm<double, 1, true>(warps_per_cta, dyn);
    return f32 ? blocks_per_sm<float, 1, false>(warps_per_cta, dyn) : blocks_per_sm<double, 1, false>(warps_per_cta, dyn);
}

size_t geodesic_team_shared_bytes(int precision, int warps_per_cta, int shared_scale) {
    return precision == CSS_FP32 ? team_smem_bytes<float>(shared_scale, warps_per_cta)
                                 : team_smem_bytes<double>(shared_scale, warps_per_cta);
}

cudaError_t launch_geodesic_team(const GeoJob& job0, const GeoJob* djobs, const GeoQueue& q, int precision,
                                 const GeoWs& ws, int warps_per_cta, int nctas, int* work_counter, int* status,
                                 unsigned long long* counters, cudaStream_t st) {
    if (warps_per_cta < 2 || warps_per_cta > MAX_TEAM) return cudaErrorInvalidValue;
    const dim3 block(32 * warps_per_cta);
    const size_t sm = geodesic_team_shared_bytes(precision, warps_per_cta, ws.shared);
    const bool light = ws.occupancy == 2, sh = ws.shared != 0;
#define CSS_LAUNCH(RT, O, S) \
    k_geodesic_team<RT, O, S><<<nctas, block, sm, st>>>(job0, djobs, q, ws, work_counter, status, counters)
    if (precision == CSS_FP32) {
        if (light) { if (sh) CSS_LAUNCH(float, 2, 1); else CSS_LAUNCH(float, 2, 0); }
        else { if (sh) CSS_LAUNCH(float, 1, 1); else CSS_LAUNCH(float, 1, 0); }
    } else {
        if (light) { if (sh) CSS_LAUNCH(double, 2, 1); else CSS_LAUNCH(double, 2, 0); }
        else { if (sh) CSS_LAUNCH(double, 1, 1); else CSS_LAUNCH(double, 1, 0); }
    }
#undef CSS_LAUNCH
    return cudaGetLastError();
}

// resident team CTAs per SM (0: the shape does not fit an SM)
template <class R, int OCC, int SH>
static int team_blocks_per_sm(int warps_per_cta, size_t dyn) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_geodesic_team<R, OCC, SH>) != cudaSuccess) { cudaGetLastError(); return 0; }
    const int room = optin - (int)fa.sharedSizeBytes;
    if (dyn > (size_t)room) return 0;
    if (cudaFuncSetAttribute(k_geodesic_team<R, OCC, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, room) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_geodesic_team<R, OCC, SH>, 32 * warps_per_cta, dyn) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

int geodesic_team_blocks_per_sm(int precision, int warps_per_cta, int shared_scale, int occupancy) {
    if (warps_per_cta < 2 || warps_per_cta > MAX_TEAM) return 0;
    const size_t dyn = geodesic_team_shared_bytes(precision, warps_per_cta, shared_scale);
    const bool f32 = precision == CSS_FP32, sh = shared_scale != 0;
    if (occupancy == 2) {
        if (sh) return f32 ? team_blocks_per_sm<float, 2, 1>(warps_per_cta, dyn) : team_blocks_per_sm<double, 2, 1>(warps_per_cta, dyn);
        return f32 ? team_blocks_per_sm<float, 2, 0>(warps_per_cta, dyn) : team_blocks_per_sm<double, 2, 0>(warps_per_cta, dyn);
    }
    if (sh) return f32 ? team_blocks_per_sm<float, 1, 1>(warps_per_cta, dyn) : team_blocks_per_sm<double, 1, 1>(warps_per_cta, dyn);
    return f32 ? team_blocks_per_sm<float, 1, 0>(warps_per_cta, dyn) : team_blocks_per_sm<double, 1, 0>(warps_per_cta, dyn);
}

cudaError_t launch_pairs_compact(int32_t n, const int32_t* pcnt, const int32_t* pj, const double* pd,
                                 const double* pt, int pair_cap, const int64_t* row_start, int32_t* out_j,
                                 double* out_d, double* out_t, cudaStream_t st) {
    k_compact<<<(n + 127) / 128, 128, 0, st>>>(n, pcnt, pj, pd, pt, pair_cap, row_start, out_j, out_d, out_t);
    return cudaGetLastError();
}

}  // namespace cssi

// =====================================================================================
// Allocation-free force evaluation.
//
// Some callers cannot call cudaMalloc at the point where they need forces: code running
// inside a host callback or a framework that forbids device allocation on its hot path,
// or an embedding that must not change the device memory footprint after start-up. For
// them css_compute_forces_noalloc runs the same neighbour/force kernel as
// css_compute_forces, but all of its scratch (the per-warp window workspace, the face
// buckets and the launch counters) lives in the one file-scope device array below, of a
// fixed size that every GPU loading this library holds until the process exits.
namespace {

constexpr size_t NA_WS_BYTES = 48ull << 20;        // per-warp window workspaces
constexpr int NA_MAX_WARPS = 1024;
constexpr int NA_WIN_CAP = 2048;                    // windows per warp
constexpr int64_t NA_MAX_FACES = 1 << 20;
constexpr int64_t NA_MAX_PARTICLES = 1 << 18;
constexpr int NA_WARPS_PER_CTA = 4;
constexpr size_t NA_OFF_GEN = NA_WS_BYTES;
constexpr size_t NA_OFF_FCNT = NA_OFF_GEN + NA_MAX_WARPS * 4;
constexpr size_t NA_OFF_FSTART = NA_OFF_FCNT + (NA_MAX_FACES + 1) * 4;
constexpr size_t NA_OFF_FITEMS = NA_OFF_FSTART + (NA_MAX_FACES + 1) * 4;
constexpr size_t NA_OFF_SCAN = NA_OFF_FITEMS + NA_MAX_PARTICLES * 4;
constexpr size_t NA_SCAN_INTS = (NA_MAX_FACES + 1) / 2048 + 2;
constexpr size_t NA_OFF_PCNT = NA_OFF_SCAN + NA_SCAN_INTS * 4;
constexpr size_t NA_OFF_SCAL = (NA_OFF_PCNT + NA_MAX_PARTICLES * 4 + 255) & ~(size_t)255;  // work, status
constexpr size_t NA_OFF_COUNT = NA_OFF_SCAL + 256;                                         // 8 counters
constexpr size_t NA_BYTES = NA_OFF_COUNT + 8 * 8;   // ~59 MB in all

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct NaDevice {
    char* base = nullptr;   // device address of g_noalloc_scratch on this device
    int layout = -1;        // precision whose workspace layout the bytes currently hold
};
NaDevice g_na[64];

// The caller's particle arrays are checked on the device before any kernel indexes with
// them: a face index outside [0, nf), or a barycentric triple that is not finite, has an
// entry below -1e-12 or does not sum to 1 within 1e-9 (the rule css_particles_set applies
// on the host), sets ST_BAD_INPUT and nothing else runs.
__global__ void k_na_validate(int32_t n, int32_t nf, const int32_t* face, const double* bary, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t f = face[i];
    const double a = bary[3 * (size_t)i], b = bary[3 * (size_t)i + 1], c = bary[3 * (size_t)i + 2];
    const bool ok = f >= 0 && f < nf && isfinite(a) && isfinite(b) && isfinite(c) && a >= -1e-12 && b >= -1e-12 &&
                    c >= -1e-12 && fabs(a + b + c - 1.0) <= 1e-9;
    if (!ok) atomicOr(status, css::ST_BAD_INPUT);
}

// the current device for the lifetime of the guard, then the caller's again
struct DeviceGuard {
    int prev = -1;
    cudaError_t set(int dev) {
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) { prev = -1; return e; }
        if (prev == dev) { prev = -1; return cudaSuccess; }
        e = cudaSetDevice(dev);
        if (e != cudaSuccess) prev = -1;
        return e;
    }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

// status bits of the kernel -> C ABI code and message
int na_status_error(css_ctx* c, int status) {
    if (status & css::ST_BAD_INPUT) {
        c->err = "compute_forces_noalloc: a face index is out of range or a barycentric triple is not finite, "
                 "non-negative and summing to 1";
        return CSS_ERR_INVALID_ARG;
    }
    if (status & (css::ST_WIN_OVERFLOW | css::ST_HASH_OVERFLOW)) {
        c->err = "compute_forces_noalloc: a source needs more than the fixed window workspace (" +
                 std::to_string(NA_WIN_CAP) + " windows per warp); use css_compute_forces";
        return CSS_ERR_QUEUE_OVERFLOW;
    }
    if (status & (css::ST_ITER_LIMIT | css::ST_WALK_LIMIT)) {
        c->err = "compute_forces_noalloc: a device loop reached its iteration cap";
        return CSS_ERR_ITER_LIMIT;
    }
    if (status & css::ST_PIECES) {
        c->err = "compute_forces_noalloc: window trimming produced too many pieces";
        return CSS_ERR_QUEUE_OVERFLOW;
    }
    c->err = "compute_forces_noalloc: device status " + std::to_string(status);
    return CSS_ERR_CUDA;
}

}  // namespace

int css_compute_forces_noalloc(const css_mesh* mesh, int64_t n, const int32_t* face, const double* bary,
                               const css_potential* pot, double r_c, int precision, double* forces,
                               double* e_pot, void* stream) {
    if (!mesh || !face || !bary || !pot || !forces || n < 1 || !(r_c > 0.0) ||
        (precision != CSS_FP64 && precision != CSS_FP32) || pot->kind < 0 || pot->kind > 2)
        return CSS_ERR_INVALID_ARG;
    css_ctx* c = mesh->ctx;
    if (n > NA_MAX_PARTICLES || mesh->nf > NA_MAX_FACES) {
        c->err = "compute_forces_noalloc: at most " + std::to_string(NA_MAX_PARTICLES) + " particles and " +
                 std::to_string(NA_MAX_FACES) + " faces fit its fixed scratch";
        return CSS_ERR_CAPACITY;
    }
    // everything runs on the device of the mesh's context, whatever device is current
    const int dev = c->device;
    if (dev < 0 || dev >= 64) return CSS_ERR_INVALID_ARG;
    DeviceGuard guard;
    cudaError_t e = guard.set(dev);
    if (e != cudaSuccess) { c->err = std::string("compute_forces_noalloc: ") + cudaGetErrorString(e); return CSS_ERR_CUDA; }
    cudaStream_t st = (cudaStream_t)stream;
    if (st) {   // a stream of another device would put these launches beside the wrong memory
        int sdev = -1;
        e = cudaStreamGetDevice(st, &sdev);
        if (e != cudaSuccess) { cudaGetLastError(); c->err = "compute_forces_noalloc: stream not usable"; return CSS_ERR_INVALID_ARG; }
        if (sdev != dev) {
            c->err = "compute_forces_noalloc: the stream belongs to device " + std::to_string(sdev) +
                     ", the mesh to device " + std::to_string(dev);
            return CSS_ERR_INVALID_ARG;
        }
    }
    NaDevice& D = g_na[dev];
    if (!D.base) {   // first call on this device: host code needs the array's device address
        e = cudaGetSymbolAddress((void**)&D.base, g_noalloc_scratch);
        if (e != cudaSuccess) { D.base = nullptr; c->err = std::string("noalloc set-up: ") + cudaGetErrorString(e); return CSS_ERR_CUDA; }
    }
    cssi::GeoWs g{};
    g.stride = cssi::geo_ws_bytes_per_warp(precision, NA_WIN_CAP, 0, &g.log_eh, &g.log_vh, &g.log_fh, &g.fcap, &g.emcap);
    g.wcap = NA_WIN_CAP;
    g.nwarps = (int)std::min<size_t>(NA_MAX_WARPS, NA_WS_BYTES / g.stride);
    g.nwarps -= g.nwarps % NA_WARPS_PER_CTA;
    g.base = D.base;
    g.gen = (uint32_t*)(D.base + NA_OFF_GEN);
    int32_t* fcnt = (int32_t*)(D.base + NA_OFF_FCNT);
    int32_t* fstart = (int32_t*)(D.base + NA_OFF_FSTART);
    int32_t* fitems = (int32_t*)(D.base + NA_OFF_FITEMS);
    int32_t* scan = (int32_t*)(D.base + NA_OFF_SCAN);
    int32_t* pcnt = (int32_t*)(D.base + NA_OFF_PCNT);
    int* scal = (int*)(D.base + NA_OFF_SCAL);
    unsigned long long* cnt = (unsigned long long*)(D.base + NA_OFF_COUNT);
    // work already queued on the context's stream (an update or a step writing the arrays
    // read here) comes first; the event was made with the context, so nothing is allocated
    e = cudaEventRecord(c->ev_order, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_order, 0);
    if (e == cudaSuccess && D.layout != precision) {
        // the array keeps the previous call's bytes; a new workspace layout starts from zero so
        // no stale bytes look like hash entries, and the face counts start from zero
        e = cudaMemsetAsync(D.base, 0, NA_OFF_FSTART, st);
        if (e == cudaSuccess) D.layout = precision;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(scal, 0, 256 + 8 * 8, st);
    int status = 0;
    // the inputs are checked before any kernel indexes with them
    if (e == cudaSuccess) {
        k_na_validate<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int32_t)n, (int32_t)mesh->nf, face, bary, scal + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, scal + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { c->err = std::string("compute_forces_noalloc: ") + cudaGetErrorString(e); return CSS_ERR_CUDA; }
    if (status) return na_status_error(c, status);
    if (e_pot) e = cudaMemsetAsync(e_pot, 0, sizeof(double), st);
    if (e == cudaSuccess)
        // the pair-count region doubles as the scatter scratch: the kernel below rewrites it
        e = cssi::launch_bucket((int32_t)n, (int32_t)mesh->nf, face, mesh->frank, fcnt, fstart, fitems, pcnt, scan, st);
    cssi::GeoJob j{};
    j.m = mesh->view();
    j.n = (int32_t)n;
    j.face = face;
    j.bary = bary;
    j.fstart = fstart;
    j.order = fitems;
    j.fitems = fitems;
    j.rc = r_c;
    j.pcnt = pcnt;
    j.want_forces = 1;
    j.pot = *pot;
    j.force = forces;
    j.epot = e_pot;
    if (e == cudaSuccess) {   // one pass, global tables; a source overflowing them is reported
        const cssi::GeoQueue q{nullptr, nullptr, (int32_t)n, nullptr, nullptr, nullptr, nullptr, 1};
        e = cssi::launch_geodesic(j, nullptr, q, precision, g, NA_WARPS_PER_CTA, g.nwarps / NA_WARPS_PER_CTA, scal,
                                  scal + 1, cnt, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, scal + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { c->err = std::string("compute_forces_noalloc: ") + cudaGetErrorString(e); return CSS_ERR_CUDA; }
    if (status) return na_status_error(c, status);
    return CSS_OK;
}
