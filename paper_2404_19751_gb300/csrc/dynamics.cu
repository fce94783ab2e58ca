// dynamics.cu -- per-step particle kernels: face bucketing, the face-walk "shift" and
// the equations of motion (Sec. 2.1 and Sec. 3.2 of the paper).
//
// Face walk (Sec. 3.2): a displacement in the tangent plane of the particle's face
// is followed across faces.  Each iteration finds, in barycentric coordinates, the
// first side the straight path meets; the particle moves there, the face changes to
// the neighbour across that side, and the rest of the displacement and every carried
// vector (velocity, orientation) are rotated into the neighbour's plane (the rigid
// unfolding map, i.e. the rotation about the shared edge).  A path through a vertex
// continues along the straightest direction, half the vertex's total angle from the
// incoming one; a boundary vertex sends the path back; an open boundary side
// reflects it.  All of it in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "css_internal.h"

namespace {

using css::DMesh;
using css::HeRec;

constexpr int WALK_MAX = 100000;
constexpr double WPI = 3.141592653589793238462643383279503;

// ------------------------------------------------------------------ exclusive scans
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class Ti, class To>
__device__ To block_excl_scan(To v, To* sh, To& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    To x = v;
    for (int o = 1; o < 32; o <<= 1) {
        To t = __shfl_up_sync(CSS_FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        To y = lane < SCAN_THREADS / 32 ? sh[lane] : (To)0;
        for (int o = 1; o < 32; o <<= 1) {
            To t = __shfl_up_sync(CSS_FULL, y, o);
            if (lane >= o) y += t;
        }
        if (lane < SCAN_THREADS / 32) sh[lane] = y;
    }
    __syncthreads();
    total = sh[SCAN_THREADS / 32 - 1];
    const To before = w > 0 ? sh[w - 1] : (To)0;
    __syncthreads();
    return before + x - v;
}

template <class Ti, class To>
__global__ void k_tile_sums(const Ti* in, int64_t n, To* sums) {
    __shared__ To sh[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    To s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) if (base + k < n) s += (To)in[base + k];
    To tot;
    block_excl_scan<Ti, To>(s, sh, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class To>
__global__ void k_scan_sums(To* sums, int nt) {
    __shared__ To sh[SCAN_THREADS / 32];
    To carry = 0;
    for (int base = 0; base < nt; base += SCAN_THREADS) {
        const int i = base + threadIdx.x;
        const To v = i < nt ? sums[i] : (To)0;
        To tot;
        const To ex = block_excl_scan<To, To>(v, sh, tot);
        if (i < nt) sums[i] = carry + ex;
        carry += tot;
    }
}

template <class Ti, class To>
__global__ void k_tile_apply(const Ti* in, int64_t n_in, int64_t n, const To* sums, To* out) {
    __shared__ To sh[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    To loc[SCAN_ITEMS];
    To s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) { loc[k] = (base + k < n_in) ? (To)in[base + k] : (To)0; s += loc[k]; }
    To tot;
    To ex = block_excl_scan<Ti, To>(s, sh, tot) + sums[blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += loc[k];
    }
}

// ------------------------------------------------------------------ bucketing (face CSR)
__global__ void k_count(int32_t n, const int32_t* face, const int32_t* frank, int32_t* cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(cnt + (frank ? frank[face[i]] : face[i]), 1);
}

// decrements the counts back to zero while placing particles
__global__ void k_scatter(int32_t n, const int32_t* face, const int32_t* frank, int32_t* cnt, const int32_t* start,
                          int32_t* items) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int f = frank ? frank[face[i]] : face[i];
    const int p = atomicSub(cnt + f, 1) - 1;
    items[start[f] + p] = i;
}

// Deterministic bucket order: the scatter above fills each face's bucket in the order its
// atomics happen to run; here each bucket is put in particle-index order.  The bucket order
// is the order in which a source meets its targets, so it fixes every force sum's order:
// runs repeat bit for bit.  A bucket of up to RANK_SCAN particles is ranked by its members
// in parallel (each counts the smaller indices, at most RANK_SCAN reads); a larger one is
// sorted by its first member alone with an in-place heap sort, O(b log b), so a crowded
// face costs no b^2 work.
constexpr int RANK_SCAN = 32;

__device__ __forceinline__ void heap_sift(int32_t* a, int root, int end) {
    const int32_t v = a[root];
    for (;;) {
        int c = 2 * root + 1;
        if (c >= end) break;
        if (c + 1 < end && a[c + 1] > a[c]) ++c;
        if (a[c] <= v) break;
        a[root] = a[c];
        root = c;
    }
    a[root] = v;
}

__device__ __forceinline__ void rank_in_bucket(int i, int key, const int32_t* start, const int32_t* tmp, int32_t* items) {
    const int st = start[key], cnt = start[key + 1] - st;
    if (cnt <= RANK_SCAN) {
        int r = 0;
        for (int q = 0; q < cnt; ++q) r += tmp[st + q] < i;
        items[st + r] = i;
        return;
    }
    if (tmp[st] != i) return;   // the bucket's first member sorts it
    int32_t* a = items + st;
    for (int q = 0; q < cnt; ++q) a[q] = tmp[st + q];
    for (int r = cnt / 2 - 1; r >= 0; --r) heap_sift(a, r, cnt);
    for (int e = cnt - 1; e > 0; --e) {
        const int32_t t = a[0];
        a[0] = a[e];
        a[e] = t;
        heap_sift(a, 0, e);
    }
}

__global__ void k_rank(int32_t n, const int32_t* face, const int32_t* frank, const int32_t* start, const int32_t* tmp,
                       int32_t* items) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    rank_in_bucket(i, frank ? frank[face[i]] : face[i], start, tmp, items);
}

// ------------------------------------------------------------------ face walk
__device__ __forceinline__ void corner(const DMesh& m, int f, int k, double& x, double& y) {
    css::face_corner(m, f, k, x, y);
}

__device__ __forceinline__ void rot(double co, double si, double& x, double& y) {
    const double a = co * x - si * y, b = si * x + co * y;
    x = a; y = b;
}

// straightest continuation through corner cw of face f (interior vertex: leave at half the
// total angle from the incoming direction; boundary vertex: turn back)
__device__ void through_vertex(const DMesh& m, int& f, int cw, double& px, double& py, double& dx, double& dy,
                               int nc, double* cx, double* cy) {
    const int v = m.fv[3 * f + cw];
    const double len = sqrt(dx * dx + dy * dy);
    const double ux = dx / len, uy = dy / len;
    double phi[2], mag[2];
    for (int q = 0; q < nc; ++q) {
        mag[q] = sqrt(cx[q] * cx[q] + cy[q] * cy[q]);
        phi[q] = atan2(ux * cy[q] - uy * cx[q], ux * cx[q] + uy * cy[q]);
    }
    double wx, wy;
    corner(m, f, cw, wx, wy);
    if (m.bnd[v]) {
        px = wx; py = wy; dx = -dx; dy = -dy;
        for (int q = 0; q < nc; ++q) { cx[q] = -cx[q]; cy[q] = -cy[q]; }
        return;
    }
    double nx, ny;
    corner(m, f, cw + 1, nx, ny);
    double ex = nx - wx, ey = ny - wy, el = sqrt(ex * ex + ey * ey);
    ex /= el; ey /= el;
    double beta = atan2(ex * (-uy) - ey * (-ux), ex * (-ux) + ey * (-uy));
    if (beta < 0.0) beta = 0.0;
    double rem = beta + 0.5 * m.theta[v];
    for (int guard = 0; guard < 64; ++guard) {
        const HeRec r = m.he[3 * f + cw];
        const double ang = atan2(r.cy, r.cx);
        if (rem <= ang) break;
        rem -= ang;
        const int hop = 3 * f + (cw == 0 ? 2 : cw - 1);
        const int tw = m.twin[hop];
        if (tw < 0) break;
        f = tw / 3;
        cw = tw - 3 * f;
    }
    corner(m, f, cw, wx, wy);
    corner(m, f, cw + 1, nx, ny);
    ex = nx - wx; ey = ny - wy; el = sqrt(ex * ex + ey * ey);
    ex /= el; ey /= el;
    double ox = ex, oy = ey;
    rot(cos(rem), sin(rem), ox, oy);
    px = wx; py = wy;
    dx = len * ox; dy = len * oy;
    for (int q = 0; q < nc; ++q) {
        double vx = ox, vy = oy;
        rot(cos(phi[q]), sin(phi[q]), vx, vy);
        cx[q] = mag[q] * vx; cy[q] = mag[q] * vy;
    }
}

// walk from (f, p) by d (face-frame components), carrying nc vectors; false on iteration cap
__device__ bool face_walk(const DMesh& m, int& f, double& px, double& py, double dx, double dy, int nc, double* cx,
                          double* cy, double* rec = nullptr, int rec_cap = 0, int* rec_n = nullptr) {
    int entry = -1;
    for (int it = 0; it < WALK_MAX; ++it) {
        const double L01 = m.lay[3 * f], x2 = m.lay[3 * f + 1], y2 = m.lay[3 * f + 2];
        double lam[3], rate[3];
        lam[2] = py / y2; lam[1] = (px - lam[2] * x2) / L01; lam[0] = 1.0 - lam[1] - lam[2];
        rate[2] = dy / y2; rate[1] = (dx - rate[2] * x2) / L01; rate[0] = -rate[1] - rate[2];
        double tmin = __longlong_as_double(0x7ff0000000000000ll);
        int imin = -1;
        for (int q = 0; q < 3; ++q) {
            if (!(rate[q] < 0.0)) continue;
            const int side = q == 2 ? 0 : q + 1;   // side opposite corner q
            if (side == entry) continue;
            double t = -lam[q] / rate[q];
            if (t < 0.0) t = 0.0;
            if (t < tmin) { tmin = t; imin = q; }
        }
        if (!(tmin < 1.0)) { px += dx; py += dy; return true; }
        const int k = imin == 2 ? 0 : imin + 1;
        const int k1 = k == 2 ? 0 : k + 1;
        const double hx = px + tmin * dx, hy = py + tmin * dy;
        double rx = (1.0 - tmin) * dx, ry = (1.0 - tmin) * dy;
        double lh[3];
        lh[2] = hy / y2; lh[1] = (hx - lh[2] * x2) / L01; lh[0] = 1.0 - lh[1] - lh[2];
        if (rec) {   // the crossing point, world position
            if (*rec_n < rec_cap) {
                const double* fr = m.frame + 9 * (size_t)f;
                for (int a = 0; a < 3; ++a) rec[3 * *rec_n + a] = fr[a] + hx * fr[3 + a] + hy * fr[6 + a];
            }
            ++*rec_n;
        }
        int vc = -1;
        if (lh[k1] < 1e-12) vc = k;
        else if (lh[k] < 1e-12) vc = k1;
        if (vc >= 0) {
            px = hx; py = hy;
            through_vertex(m, f, vc, px, py, rx, ry, nc, cx, cy);
            dx = rx; dy = ry; entry = -1;
            continue;
        }
        const int h = 3 * f + k;
        const int tw = m.twin[h];
        double ax, ay, bx, by;
        corner(m, f, k, ax, ay);
        corner(m, f, k1, bx, by);
        const double L = m.he[h].L;
        const double ux = (bx - ax) / L, uy = (by - ay) / L;
        if (tw < 0) {
            const double pr = rx * ux + ry * uy;
            rx = 2.0 * pr * ux - rx; ry = 2.0 * pr * uy - ry;
            for (int q = 0; q < nc; ++q) {
                const double pc = cx[q] * ux + cy[q] * uy;
                cx[q] = 2.0 * pc * ux - cx[q]; cy[q] = 2.0 * pc * uy - cy[q];
            }
            px = hx; py = hy; dx = rx; dy = ry; entry = k;
            continue;
        }
        const int g = tw / 3, k2 = tw - 3 * g;
        double qax, qay, qbx, qby;
        corner(m, g, k2 + 1, qax, qay);   // image of corner k
        corner(m, g, k2, qbx, qby);       // image of corner k+1
        const double Lg = sqrt((qbx - qax) * (qbx - qax) + (qby - qay) * (qby - qay));
        const double vx = (qbx - qax) / Lg, vy = (qby - qay) / Lg;
        const double co = ux * vx + uy * vy, si = ux * vy - uy * vx;
        double ox = hx - ax, oy = hy - ay;
        rot(co, si, ox, oy);
        px = qax + ox; py = qay + oy;
        rot(co, si, rx, ry);
        for (int q = 0; q < nc; ++q) rot(co, si, cx[q], cy[q]);
        dx = rx; dy = ry; f = g; entry = k2;
    }
    return false;
}

__device__ __forceinline__ void to_face(const DMesh& m, int f, const double* v, double& x, double& y) {
    const double* fr = m.frame + 9 * (size_t)f;
    x = v[0] * fr[3] + v[1] * fr[4] + v[2] * fr[5];
    y = v[0] * fr[6] + v[1] * fr[7] + v[2] * fr[8];
}
__device__ __forceinline__ void to_world(const DMesh& m, int f, double x, double y, double* v) {
    const double* fr = m.frame + 9 * (size_t)f;
    v[0] = x * fr[3] + y * fr[6];
    v[1] = x * fr[4] + y * fr[7];
    v[2] = x * fr[5] + y * fr[8];
}

__device__ bool shift_particle(const DMesh& m, int& f, double* bary, const double* d3, int nc, double* c3a,
                               double* c3b) {
    double px = bary[1] * m.lay[3 * f] + bary[2] * m.lay[3 * f + 1];
    double py = bary[2] * m.lay[3 * f + 2];
    double dx, dy, cx[2], cy[2];
    to_face(m, f, d3, dx, dy);
    if (nc > 0) to_face(m, f, c3a, cx[0], cy[0]);
    if (nc > 1) to_face(m, f, c3b, cx[1], cy[1]);
    const bool ok = face_walk(m, f, px, py, dx, dy, nc, cx, cy);
    const double L01 = m.lay[3 * f], x2 = m.lay[3 * f + 1], y2 = m.lay[3 * f + 2];
    double l2 = py / y2, l1 = (px - l2 * x2) / L01, l0 = 1.0 - l1 - l2;
    l0 = l0 < 0.0 ? 0.0 : l0; l1 = l1 < 0.0 ? 0.0 : l1; l2 = l2 < 0.0 ? 0.0 : l2;
    const double s = l0 + l1 + l2;
    bary[0] = l0 / s; bary[1] = l1 / s; bary[2] = l2 / s;
    if (nc > 0) to_world(m, f, cx[0], cy[0], c3a);
    if (nc > 1) to_world(m, f, cx[1], cy[1], c3b);
    return ok;
}

__device__ __forceinline__ void clamp_disp(double* d, double maxd) {
    const double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (n > maxd) { const double s = maxd / n; d[0] *= s; d[1] *= s; d[2] *= s; }
}

// ------------------------------------------------------------------ Philox4x32-10 (Salmon et al., SC'11)
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        const uint32_t a0 = c[0], a2 = c[2];
        const uint32_t hi0 = __umulhi(0xD2511F53u, a0), lo0 = 0xD2511F53u * a0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, a2), lo1 = 0xCD9E8D57u * a2;
        c[0] = hi1 ^ c[1] ^ k0;
        c[1] = lo1;
        c[2] = hi0 ^ c[3] ^ k1;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ void normal_pair(uint64_t seed, uint64_t particle, uint64_t step, double& z0, double& z1) {
    uint32_t c[4] = {(uint32_t)particle, (uint32_t)(particle >> 32), (uint32_t)step, (uint32_t)(step >> 32)};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6) + 0.5) / 9007199254740992.0;
    const double u2 = ((double)(c[2] >> 5) * 67108864.0 + (double)(c[3] >> 6) + 0.5) / 9007199254740992.0;
    const double r = sqrt(-2.0 * log(u1));
    z0 = r * cos(2.0 * WPI * u2);
    z1 = r * sin(2.0 * WPI * u2);
}

// ------------------------------------------------------------------ integrators
// first half kick and drift of particle i (velocity Verlet, Sec. 2.1)
__device__ void kick_drift_one(const DMesh& m, int i, int32_t* face, double* bary, double* vel, const double* force,
                               const css_integrator& it, int* status) {
    const double h = 0.5 * it.dt / it.mass;
    double v[3], d[3];
    for (int a = 0; a < 3; ++a) { v[a] = vel[3 * i + a] + h * force[3 * i + a]; d[a] = it.dt * v[a]; }
    clamp_disp(d, it.max_disp);
    int f = face[i];
    double b[3] = {bary[3 * i], bary[3 * i + 1], bary[3 * i + 2]};
    if (!shift_particle(m, f, b, d, 1, v, nullptr)) atomicOr(status, css::ST_WALK_LIMIT);
    face[i] = f;
    for (int a = 0; a < 3; ++a) { bary[3 * i + a] = b[a]; vel[3 * i + a] = v[a]; }
}
__global__ void k_nve_kick_drift(DMesh m, int32_t n, int32_t* face, double* bary, double* vel, const double* force,
                                 css_integrator it, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) kick_drift_one(m, i, face, bary, vel, force, it, status);
}

__global__ void k_nve_kick(int32_t n, double* vel, const double* force, double h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    vel[i] += h * force[i];
}

// overdamped (Brownian or active) move of particle i (Sec. 2.1)
__device__ void overdamped_one(const DMesh& m, int i, int32_t* face, double* bary, double* orient, const double* force,
                               const css_integrator& it, uint64_t seed, const int64_t* dstep, const double* noise,
                               int* status) {
    double z0 = 0.0, z1 = 0.0;   // steepest descent draws no noise
    if (it.kind != CSS_INT_GD) {
        if (noise) { z0 = noise[2 * (size_t)i]; z1 = noise[2 * (size_t)i + 1]; }
        else normal_pair(seed, (uint64_t)i, (uint64_t)*dstep, z0, z1);
    }
    int f = face[i];
    const double* fr = m.frame + 9 * (size_t)f;
    double b[3] = {bary[3 * i], bary[3 * i + 1], bary[3 * i + 2]};
    double d[3];
    bool ok;
    if (it.kind == CSS_INT_BD || it.kind == CSS_INT_GD) {
        const double amp = it.kind == CSS_INT_BD ? sqrt(2.0 * it.kT * it.dt / it.lambda) : 0.0;
        for (int a = 0; a < 3; ++a) d[a] = it.dt / it.lambda * force[3 * i + a] + amp * (z0 * fr[3 + a] + z1 * fr[6 + a]);
        clamp_disp(d, it.max_disp);
        ok = shift_particle(m, f, b, d, 0, nullptr, nullptr);
    } else {
        double o[3] = {orient[3 * i], orient[3 * i + 1], orient[3 * i + 2]};
        for (int a = 0; a < 3; ++a) d[a] = it.dt * (it.v0 * o[a] + force[3 * i + a] / it.lambda);
        clamp_disp(d, it.max_disp);
        ok = shift_particle(m, f, b, d, 1, o, nullptr);
        double ox, oy;
        to_face(m, f, o, ox, oy);
        const double on = sqrt(ox * ox + oy * oy);
        ox /= on; oy /= on;
        const double ang = sqrt(2.0 * it.Dr * it.dt) * z0;
        rot(cos(ang), sin(ang), ox, oy);
        to_world(m, f, ox, oy, o);
        for (int a = 0; a < 3; ++a) orient[3 * i + a] = o[a];
    }
    if (!ok) atomicOr(status, css::ST_WALK_LIMIT);
    face[i] = f;
    for (int a = 0; a < 3; ++a) bary[3 * i + a] = b[a];
}
__global__ void k_overdamped(DMesh m, int32_t n, int32_t* face, double* bary, double* orient, const double* force,
                             css_integrator it, uint64_t seed, const int64_t* dstep, const double* noise, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) overdamped_one(m, i, face, bary, orient, force, it, seed, dstep, noise, status);
}

__global__ void k_step_inc(int64_t* dstep) { *dstep += 1; }

// bitwise comparison of an uploaded state with the current one: bit 1 = positions (face or
// barycentrics) differ, bit 2 = velocities differ; arrays the caller did not upload are NULL
__global__ void k_state_diff(int32_t n, const int32_t* nf, const int32_t* of, const double* nb, const double* ob,
                             const double* nv, const double* ov, int* flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int d = 0;
    if (nf && nf[i] != of[i]) d |= 1;
    for (int a = 0; a < 3; ++a) {
        if (nb && __double_as_longlong(nb[3 * i + a]) != __double_as_longlong(ob[3 * i + a])) d |= 1;
        if (nv && __double_as_longlong(nv[3 * i + a]) != __double_as_longlong(ov[3 * i + a])) d |= 2;
    }
    if (d) atomicOr(flag, d);
}

// ------------------------------------------------------------------ path polylines
// Path p: the straightest walk from particle src[p] along the world tangent tan[p] for
// length len[p], recorded as world points (start, each crossing, end; at most cap).
__global__ void k_trace(DMesh m, int64_t npaths, const int32_t* pface, const double* pbary, const int32_t* src,
                        const double* tan, const double* len, int cap, double* pts, int32_t* npts,
                        int32_t* end_face, double* end_bary, int* status) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= npaths) return;
    const int i = src[p];
    int f = pface[i];
    double b[3] = {pbary[3 * (size_t)i], pbary[3 * (size_t)i + 1], pbary[3 * (size_t)i + 2]};
    double* out = pts + 3 * (size_t)p * cap;
    double px = b[1] * m.lay[3 * f] + b[2] * m.lay[3 * f + 1], py = b[2] * m.lay[3 * f + 2];
    if (cap > 0) {
        const double* fr = m.frame + 9 * (size_t)f;
        for (int a = 0; a < 3; ++a) out[a] = fr[a] + px * fr[3 + a] + py * fr[6 + a];
    }
    double d3[3] = {len[p] * tan[3 * p], len[p] * tan[3 * p + 1], len[p] * tan[3 * p + 2]};
    double dx, dy;
    to_face(m, f, d3, dx, dy);
    int n = 0;
    const bool ok = face_walk(m, f, px, py, dx, dy, 0, nullptr, nullptr, cap > 1 ? out + 3 : out, cap > 1 ? cap - 1 : 0, &n);
    if (!ok) atomicOr(status, css::ST_WALK_LIMIT);
    n += 1;
    if (n < cap) {
        const double* fr = m.frame + 9 * (size_t)f;
        for (int a = 0; a < 3; ++a) out[3 * n + a] = fr[a] + px * fr[3 + a] + py * fr[6 + a];
    }
    npts[p] = n + 1;
    const double L01 = m.lay[3 * f], x2 = m.lay[3 * f + 1], y2 = m.lay[3 * f + 2];
    double l2 = py / y2, l1 = (px - l2 * x2) / L01, l0 = 1.0 - l1 - l2;
    l0 = l0 < 0.0 ? 0.0 : l0; l1 = l1 < 0.0 ? 0.0 : l1; l2 = l2 < 0.0 ? 0.0 : l2;
    const double sb = l0 + l1 + l2;
    end_face[p] = f;
    end_bary[3 * p] = l0 / sb; end_bary[3 * p + 1] = l1 / sb; end_bary[3 * p + 2] = l2 / sb;
}

// ------------------------------------------------------------------ FIRE minimiser
// Device state of one set: [0] step, [1] alpha, [2] consecutive steps with P > 0,
// [3] velocity factor, [4] force factor of the mixing, [5..7] sums P, |v|^2, |F|^2.
constexpr double FIRE_ALPHA0 = 0.1, FIRE_FINC = 1.1, FIRE_FDEC = 0.5, FIRE_FALPHA = 0.99;
constexpr int FIRE_NMIN = 5;

__global__ void k_fire_reduce(int64_t n3, const double* vel, const double* force, double* st) {
    double P = 0.0, vv = 0.0, ff = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = vel[i], f = force[i];
        P += f * v;
        vv += v * v;
        ff += f * f;
    }
    P = css::warp_sum(P);
    vv = css::warp_sum(vv);
    ff = css::warp_sum(ff);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(st + 5, P);
        atomicAdd(st + 6, vv);
        atomicAdd(st + 7, ff);
    }
}

// one thread: the mixing factors with the current alpha, then the step / alpha update
__global__ void k_fire_control(double* st, double dt_max) {
    const double P = st[5], vv = st[6], ff = st[7], alpha = st[1];
    double c1 = 1.0, c2 = 0.0;
    if (ff > 0.0) { c1 = 1.0 - alpha; c2 = alpha * sqrt(vv) / sqrt(ff); }
    if (P > 0.0) {
        st[2] += 1.0;
        if (st[2] > FIRE_NMIN) {
            st[0] = fmin(st[0] * FIRE_FINC, dt_max);
            st[1] = alpha * FIRE_FALPHA;
        }
    } else {
        st[2] = 0.0;
        st[0] *= FIRE_FDEC;
        st[1] = FIRE_ALPHA0;
        c1 = 0.0;
        c2 = 0.0;
    }
    st[3] = c1;
    st[4] = c2;
    st[5] = st[6] = st[7] = 0.0;
}

__global__ void k_fire_mix_kick_drift(DMesh m, int32_t n, int32_t* face, double* bary, double* vel,
                                      const double* force, const double* st, css_integrator it, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c1 = st[3], c2 = st[4], dt = st[0], h = 0.5 * dt / it.mass;
    double v[3], d[3];
    for (int a = 0; a < 3; ++a) {
        v[a] = c1 * vel[3 * i + a] + c2 * force[3 * i + a];
        v[a] += h * force[3 * i + a];
        d[a] = dt * v[a];
    }
    clamp_disp(d, it.max_disp);
    int f = face[i];
    double b[3] = {bary[3 * i], bary[3 * i + 1], bary[3 * i + 2]};
    if (!shift_particle(m, f, b, d, 1, v, nullptr)) atomicOr(status, css::ST_WALK_LIMIT);
    face[i] = f;
    for (int a = 0; a < 3; ++a) { bary[3 * i + a] = b[a]; vel[3 * i + a] = v[a]; }
}

__global__ void k_fire_kick(int64_t n3, double* vel, const double* force, const double* st, double mass) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n3) vel[i] += 0.5 * st[0] / mass * force[i];
}

// ------------------------------------------------------------------ many sets in one launch
// Work item k of a batch belongs to the set s with offs[s] <= k < offs[s+1] (a handful of
// bisection steps over the set offsets) and is that set's particle k - offs[s].
__device__ __forceinline__ int set_of(const int32_t* offs, int nsets, int k) {
    int lo = 0, hi = nsets;   // offs[lo] <= k < offs[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offs[mid] <= k) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_batch_kick_drift(const cssi::SetView* sv, const int32_t* offs, int nsets, css_integrator it,
                                   int* status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= offs[nsets]) return;
    const int s = set_of(offs, nsets, k);
    const cssi::SetView& V = sv[s];
    kick_drift_one(V.m, k - offs[s], V.face, V.bary, V.vel, V.force, it, status);
}

__global__ void k_batch_kick(const cssi::SetView* sv, const int32_t* offs, int nsets, double h) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= offs[nsets]) return;
    const int s = set_of(offs, nsets, k);
    const int i = k - offs[s];
    double* v = sv[s].vel + 3 * (size_t)i;
    const double* f = sv[s].force + 3 * (size_t)i;
    v[0] += h * f[0];
    v[1] += h * f[1];
    v[2] += h * f[2];
}

__global__ void k_batch_overdamped(const cssi::SetView* sv, const int32_t* offs, int nsets, css_integrator it,
                                   int* status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= offs[nsets]) return;
    const int s = set_of(offs, nsets, k);
    const cssi::SetView& V = sv[s];
    overdamped_one(V.m, k - offs[s], V.face, V.bary, V.orient, V.force, it, V.seed, V.dstep, nullptr, status);
}

__global__ void k_batch_step_inc(const cssi::SetView* sv, int nsets) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsets) *sv[s].dstep += 1;
}

__global__ void k_batch_count(const cssi::SetView* sv, const int32_t* offs, int nsets) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= offs[nsets]) return;
    const int s = set_of(offs, nsets, k);
    const cssi::SetView& V = sv[s];
    const int f = V.face[k - offs[s]];
    atomicAdd(V.fcnt + (V.m.frank ? V.m.frank[f] : f), 1);
}

// one block per set: exclusive scan of its nf + 1 face counts (the last count is zero)
__global__ void __launch_bounds__(SCAN_THREADS) k_batch_scan(const cssi::SetView* sv) {
    __shared__ int32_t sh[SCAN_THREADS / 32];
    const cssi::SetView& V = sv[blockIdx.x];
    const int64_t n = (int64_t)V.m.nf + 1;
    int32_t carry = 0;
    for (int64_t base = 0; base < n; base += SCAN_THREADS) {
        const int64_t i = base + threadIdx.x;
        const int32_t v = i < V.m.nf ? V.fcnt[i] : 0;
        int32_t total = 0;
        const int32_t ex = block_excl_scan<int32_t, int32_t>(v, sh, total);
        if (i < n) V.fstart[i] = carry + ex;
        carry += total;
    }
}

__global__ void k_batch_scatter(const cssi::SetView* sv, const int32_t* offs, int nsets) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= offs[nsets]) return;
    const int s = set_of(offs, nsets, k);
    const cssi::SetView& V = sv[s];
    const int i = k - offs[s];
    const int f = V.face[i];
    const int key = V.m.frank ? V.m.frank[f] : f;
    const int p = atomicSub(V.fcnt + key, 1) - 1;
    V.ftmp[V.fstart[key] + p] = i;
}
__global__ void k_batch_rank(const cssi::SetView* sv, const int32_t* offs, int nsets) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= offs[nsets]) return;
    const int s = set_of(offs, nsets, k);
    const cssi::SetView& V = sv[s];
    const int i = k - offs[s];
    const int f = V.face[i];
    rank_in_bucket(i, V.m.frank ? V.m.frank[f] : f, V.fstart, V.ftmp, V.fitems);
}


inline unsigned nb(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

namespace cssi {

size_t scan_tmp_ints(int64_t count) { return (size_t)((count + SCAN_TILE - 1) / SCAN_TILE) + 1; }

cudaError_t launch_scan_i32(const int32_t* in, int32_t* out_excl, int64_t count, int32_t* tmp, cudaStream_t st) {
    const int nt = (int)((count + SCAN_TILE - 1) / SCAN_TILE);
    k_tile_sums<int32_t, int32_t><<<nt, SCAN_THREADS, 0, st>>>(in, count, tmp);
    k_scan_sums<int32_t><<<1, SCAN_THREADS, 0, st>>>(tmp, nt);
    k_tile_apply<int32_t, int32_t><<<nt, SCAN_THREADS, 0, st>>>(in, count, count, tmp, out_excl);
    return cudaGetLastError();
}

// row_start[0..n] (int64) from n counts: the tile sums live at the end of row_start's
// scratch tail, so the caller passes row_start with n + 1 + scan_tmp_ints(n + 1) slots
cudaError_t launch_scan_rows(const int32_t* cnt, int64_t* row_start, int32_t n, cudaStream_t st) {
    const int64_t count = (int64_t)n + 1;
    const int nt = (int)((count + SCAN_TILE - 1) / SCAN_TILE);
    int64_t* tmp = row_start + count;
    k_tile_sums<int32_t, int64_t><<<nt, SCAN_THREADS, 0, st>>>(cnt, n, tmp);
    k_scan_sums<int64_t><<<1, SCAN_THREADS, 0, st>>>(tmp, nt);
    k_tile_apply<int32_t, int64_t><<<nt, SCAN_THREADS, 0, st>>>(cnt, n, count, tmp, row_start);
    return cudaGetLastError();
}

cudaError_t launch_bucket(int32_t n, int32_t nf, const int32_t* face, const int32_t* frank, int32_t* fcnt,
                          int32_t* fstart, int32_t* fitems, int32_t* ftmp, int32_t* scan_tmp, cudaStream_t st) {
    k_count<<<nb(n), 256, 0, st>>>(n, face, frank, fcnt);
    cudaError_t e = launch_scan_i32(fcnt, fstart, (int64_t)nf + 1, scan_tmp, st);
    if (e != cudaSuccess) return e;
    k_scatter<<<nb(n), 256, 0, st>>>(n, face, frank, fcnt, fstart, ftmp);
    k_rank<<<nb(n), 256, 0, st>>>(n, face, frank, fstart, ftmp, fitems);
    return cudaGetLastError();
}

cudaError_t launch_nve_kick_drift(const DMesh& m, int32_t n, int32_t* face, double* bary, double* vel,
                                  const double* force, css_integrator it, int* status, cudaStream_t st) {
    k_nve_kick_drift<<<nb(n, 128), 128, 0, st>>>(m, n, face, bary, vel, force, it, status);
    return cudaGetLastError();
}

cudaError_t launch_nve_kick(int32_t n, double* vel, const double* force, css_integrator it, cudaStream_t st) {
    k_nve_kick<<<nb(3 * (int64_t)n), 256, 0, st>>>(n, vel, force, 0.5 * it.dt / it.mass);
    return cudaGetLastError();
}

cudaError_t launch_overdamped_move(const DMesh& m, int32_t n, int32_t* face, double* bary, double* orient,
                                   const double* force, css_integrator it, uint64_t seed, const int64_t* dstep,
                                   const double* noise, int* status, cudaStream_t st) {
    k_overdamped<<<nb(n, 128), 128, 0, st>>>(m, n, face, bary, orient, force, it, seed, dstep, noise, status);
    return cudaGetLastError();
}

cudaError_t launch_step_inc(int64_t* dstep, cudaStream_t st) {
    k_step_inc<<<1, 1, 0, st>>>(dstep);
    return cudaGetLastError();
}

cudaError_t launch_fire_move(const DMesh& m, int32_t n, int32_t* face, double* bary, double* vel,
                             const double* force, double* fire_state, css_integrator it, int half, int* status,
                             cudaStream_t st) {
    if (half == 0) {
        const int64_t n3 = 3 * (int64_t)n;
        k_fire_reduce<<<(unsigned)std::min<int64_t>(nb(n3), 1024), 256, 0, st>>>(n3, vel, force, fire_state);
        k_fire_control<<<1, 1, 0, st>>>(fire_state, 10.0 * it.dt);
        k_fire_mix_kick_drift<<<nb(n, 128), 128, 0, st>>>(m, n, face, bary, vel, force, fire_state, it, status);
    } else {
        k_fire_kick<<<nb(3 * (int64_t)n), 256, 0, st>>>(3 * (int64_t)n, vel, force, fire_state, it.mass);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ shortest-path legs (Sec. 2.2)
// A shortest path is a chain of straight legs meeting at pseudo-source vertices; the
// neighbour kernel's path instantiation records, for every pair, each leg's start node,
// direction and length.  Here every leg is walked straight across the faces it crosses.

__device__ __forceinline__ double corner_angle(const DMesh& m, int f, int k) {
    const HeRec& r = m.he[3 * f + k];
    return atan2(r.cy, r.cx);
}

// The face of the ring of the vertex at corner k of face f whose wedge holds the direction
// at angle phi counted counter-clockwise from the edge corner k -> k+1 (negative: clockwise
// of it; beyond the corner angle: past the edge corner k -> k+2).  On success f, k and phi
// refer to that face, phi clamped into its wedge; false when the direction leaves the ring
// through a boundary edge.
__device__ bool ring_locate(const DMesh& m, int& f, int& k, double& phi) {
    const double tol = 1e-12;
    for (int guard = 0; guard < 256; ++guard) {
        const double a = corner_angle(m, f, k);
        if (phi < -tol) {
            const int tw = m.twin[3 * f + k];                       // across corner k -> k+1
            if (tw < 0) return false;
            f = tw / 3;
            const int kt = tw - 3 * f;
            k = kt == 2 ? 0 : kt + 1;
            phi += corner_angle(m, f, k);
        } else if (phi > a + tol) {
            const int tw = m.twin[3 * f + (k == 0 ? 2 : k - 1)];    // across corner k+2 -> k
            if (tw < 0) return false;
            phi -= a;
            f = tw / 3;
            k = tw - 3 * f;
        } else {
            phi = phi < 0.0 ? 0.0 : (phi > a ? a : phi);
            return true;
        }
    }
    return false;
}

__device__ void corner_dir(const DMesh& m, int f, int k, double phi, double& dx, double& dy) {
    double ax, ay, bx, by;
    corner(m, f, k, ax, ay);
    corner(m, f, k + 1, bx, by);
    const double L = sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
    dx = (bx - ax) / L;
    dy = (by - ay) / L;
    rot(cos(phi), sin(phi), dx, dy);
}

// A leg meets a vertex on its way and goes on straight: at angle pi from the reversed
// incoming direction, counter-clockwise around the ring if it holds that angle on that
// side, else clockwise (a boundary vertex holds it on one side only).
__device__ bool vertex_pass(const DMesh& m, int& f, int& k, double& dx, double& dy) {
    double ax, ay, bx, by;
    corner(m, f, k, ax, ay);
    corner(m, f, k + 1, bx, by);
    const double L = sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
    const double ex = (bx - ax) / L, ey = (by - ay) / L;
    double beta = atan2(ex * (-dy) - ey * (-dx), ex * (-dx) + ey * (-dy));
    const double a = corner_angle(m, f, k);
    beta = beta < 0.0 ? 0.0 : (beta > a ? a : beta);
    int g = f, kg = k;
    double phi = beta + WPI;
    if (!ring_locate(m, g, kg, phi)) {
        g = f; kg = k; phi = beta - WPI;
        if (!ring_locate(m, g, kg, phi)) return false;
    }
    f = g;
    k = kg;
    corner_dir(m, g, kg, phi, dx, dy);
    return true;
}

__device__ __forceinline__ void layout_world(const DMesh& m, int f, double x, double y, double* w) {
    const double* fr = m.frame + 9 * (size_t)f;
    for (int a = 0; a < 3; ++a) w[a] = fr[a] + x * fr[3 + a] + y * fr[6 + a];
}

__device__ __forceinline__ void wrap_world(const DMesh& m, double* w) {
    if (m.periodic)
        for (int a = 0; a < 2; ++a) w[a] -= m.per[a] * floor(w[a] / m.per[a]);
}

// One leg: from corner kc of face f (kc < 3; the unit direction (dx, dy) of f's layout may
// point into any face of the vertex's ring) or from the point (px, py) of f (kc == 3), for
// length len.  Writes the world position (wrapped into the period) of every edge or vertex
// crossed before the end to rec (at most cap; *nrec counts all) and returns the end point
// (face f, layout point px, py).  A crossing within 1e-12 of the leg's end is the end.
// Returns 0, or a negative code (ring left through the boundary, boundary crossed, no end).
__device__ int leg_walk(const DMesh& m, int& f, int kc, double& px, double& py, double dx, double dy, double len,
                        double* rec, int cap, int& nrec) {
    int cn = kc < 3 ? kc : -1;
    if (cn < 0) {   // a start point on a corner of its face starts from that vertex
        const double L01 = m.lay[3 * f], x2 = m.lay[3 * f + 1], y2 = m.lay[3 * f + 2];
        const double l2 = py / y2, l1 = (px - l2 * x2) / L01, l0 = 1.0 - l1 - l2;
        if (l0 > 1.0 - 1e-12) cn = 0;
        if (l1 > 1.0 - 1e-12) cn = 1;
        if (l2 > 1.0 - 1e-12) cn = 2;
    }
    if (cn >= 0) {
        double ax, ay, bx, by;
        corner(m, f, cn, ax, ay);
        corner(m, f, cn + 1, bx, by);
        const double L = sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
        const double ux = (bx - ax) / L, uy = (by - ay) / L;
        double phi = atan2(ux * dy - uy * dx, ux * dx + uy * dy);
        if (!ring_locate(m, f, cn, phi)) return -3;
        corner_dir(m, f, cn, phi, dx, dy);
        corner(m, f, cn, px, py);
    }
    double rem = len;
    int entry = -1;
    for (int it = 0; it < WALK_MAX; ++it) {
        const double L01 = m.lay[3 * f], x2 = m.lay[3 * f + 1], y2 = m.lay[3 * f + 2];
        const double Dx = dx * rem, Dy = dy * rem;
        double lam[3], rate[3];
        lam[2] = py / y2; lam[1] = (px - lam[2] * x2) / L01; lam[0] = 1.0 - lam[1] - lam[2];
        rate[2] = Dy / y2; rate[1] = (Dx - rate[2] * x2) / L01; rate[0] = -rate[1] - rate[2];
        double tmin = __longlong_as_double(0x7ff0000000000000ll);
        int imin = -1;
        for (int q = 0; q < 3; ++q) {
            if (cn >= 0 && q != cn) continue;   // from a corner: only the far edge
            if (!(rate[q] < 0.0)) continue;
            const int side = q == 2 ? 0 : q + 1;
            if (side == entry) continue;
            double t = -lam[q] / rate[q];
            if (t < 0.0) t = 0.0;
            if (t < tmin) { tmin = t; imin = q; }
        }
        if (!(tmin < 1.0 - 1e-12)) { px += Dx; py += Dy; return 0; }
        const int k = imin == 2 ? 0 : imin + 1;
        const int k1 = k == 2 ? 0 : k + 1;
        const double hx = px + tmin * Dx, hy = py + tmin * Dy;
        rem *= (1.0 - tmin);
        double lh[3];
        lh[2] = hy / y2; lh[1] = (hx - lh[2] * x2) / L01; lh[0] = 1.0 - lh[1] - lh[2];
        int vc = -1;
        if (lh[k1] < 1e-12) vc = k;
        else if (lh[k] < 1e-12) vc = k1;
        if (rec && nrec < cap) {
            double w[3];
            if (vc >= 0) { double vx, vy; corner(m, f, vc, vx, vy); layout_world(m, f, vx, vy, w); }
            else layout_world(m, f, hx, hy, w);
            wrap_world(m, w);
            for (int a = 0; a < 3; ++a) rec[3 * nrec + a] = w[a];
        }
        ++nrec;
        if (vc >= 0) {
            int kk = vc;
            if (!vertex_pass(m, f, kk, dx, dy)) return -4;
            cn = kk;
            corner(m, f, cn, px, py);
            entry = -1;
            continue;
        }
        const int h = 3 * f + k;
        const int tw = m.twin[h];
        if (tw < 0) return -5;   // a shortest path never crosses the boundary
        double ax, ay, bx, by;
        corner(m, f, k, ax, ay);
        corner(m, f, k1, bx, by);
        const double L = sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
        const double ux = (bx - ax) / L, uy = (by - ay) / L;
        const int g = tw / 3, k2 = tw - 3 * g;
        double qax, qay, qbx, qby;
        corner(m, g, k2 + 1, qax, qay);
        corner(m, g, k2, qbx, qby);
        const double Lg = sqrt((qbx - qax) * (qbx - qax) + (qby - qay) * (qby - qay));
        const double vx = (qbx - qax) / Lg, vy = (qby - qay) / Lg;
        const double co = ux * vx + uy * vy, si = ux * vy - uy * vx;
        double ox = hx - ax, oy = hy - ay;
        rot(co, si, ox, oy);
        px = qax + ox; py = qay + oy;
        rot(co, si, dx, dy);
        f = g; entry = k2; cn = -1;
    }
    return -2;
}

// world position (wrapped) of a path node: 4 * face + corner, or (fk < 0) particle pi
__device__ void node_world(const DMesh& m, int fk, int pi, const int32_t* pface, const double* pbary, double* w) {
    if (fk >= 0) {
        double x, y;
        corner(m, fk >> 2, fk & 3, x, y);
        layout_world(m, fk >> 2, x, y, w);
    } else {
        const int f = pface[pi];
        const double* b = pbary + 3 * (size_t)pi;
        layout_world(m, f, b[1] * m.lay[3 * f] + b[2] * m.lay[3 * f + 1], b[2] * m.lay[3 * f + 2], w);
    }
    wrap_world(m, w);
}

// Leg l starts at node start_fk[l] (4 * face + corner; corner 3: the point of particle
// start_pi[l] in that face), goes along dir[l] for len[l], and must end on node next_fk[l]
// (or, if negative, on particle next_pi[l]).  Writes its start, crossings and that next
// node (world, wrapped), and gap[l] = distance between its end and the next node.
__global__ void k_legs(DMesh m, int64_t nleg, const int32_t* pface, const double* pbary, const int32_t* start_fk,
                       const int32_t* start_pi, const double* dir, const double* len, const int32_t* next_fk,
                       const int32_t* next_pi, int cap, double* rec, int32_t* nrec, double* start_w,
                       double* next_w, double* gap) {
    const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= nleg) return;
    const int fk = start_fk[l];
    int f = fk >> 2;
    const int kc = fk & 3;
    double px, py;
    if (kc < 3) corner(m, f, kc, px, py);
    else {
        const double* b = pbary + 3 * (size_t)start_pi[l];
        px = b[1] * m.lay[3 * f] + b[2] * m.lay[3 * f + 1];
        py = b[2] * m.lay[3 * f + 2];
    }
    node_world(m, kc < 3 ? fk : -1, start_pi[l], pface, pbary, start_w + 3 * l);
    int n = 0;
    const int rc = leg_walk(m, f, kc, px, py, dir[2 * l], dir[2 * l + 1], len[l], rec + 3 * (size_t)l * cap, cap, n);
    double e[3], q[3];
    layout_world(m, f, px, py, e);
    node_world(m, next_fk[l], next_pi[l], pface, pbary, q);
    for (int a = 0; a < 3; ++a) next_w[3 * l + a] = q[a];
    double d[3] = {e[0] - q[0], e[1] - q[1], e[2] - q[2]};
    if (m.periodic)
        for (int a = 0; a < 2; ++a) d[a] -= m.per[a] * floor(d[a] / m.per[a] + 0.5);
    gap[l] = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    nrec[l] = rc < 0 ? rc : n;
}

cudaError_t launch_trace(const DMesh& m, int64_t npaths, const int32_t* pface, const double* pbary,
                         const int32_t* src, const double* tan, const double* len, int cap, double* pts,
                         int32_t* npts, int32_t* end_face, double* end_bary, int* status, cudaStream_t st) {
    if (npaths < 1) return cudaSuccess;
    k_trace<<<nb(npaths, 128), 128, 0, st>>>(m, npaths, pface, pbary, src, tan, len, cap, pts, npts, end_face,
                                              end_bary, status);
    return cudaGetLastError();
}

cudaError_t launch_legs(const DMesh& m, int64_t nleg, const int32_t* pface, const double* pbary,
                        const int32_t* start_fk, const int32_t* start_pi, const double* dir, const double* len,
                        const int32_t* next_fk, const int32_t* next_pi, int cap, double* rec, int32_t* nrec,
                        double* start_w, double* next_w, double* gap, cudaStream_t st) {
    if (nleg < 1) return cudaSuccess;
    k_legs<<<nb(nleg, 128), 128, 0, st>>>(m, nleg, pface, pbary, start_fk, start_pi, dir, len, next_fk, next_pi, cap,
                                          rec, nrec, start_w, next_w, gap);
    return cudaGetLastError();
}

cudaError_t launch_state_diff(int32_t n, const int32_t* new_f, const int32_t* old_f, const double* new_b,
                              const double* old_b, const double* new_v, const double* old_v, int* flag, cudaStream_t st) {
    if (n > 0) k_state_diff<<<nb(n), 256, 0, st>>>(n, new_f, old_f, new_b, old_b, new_v, old_v, flag);
    return cudaGetLastError();
}

cudaError_t launch_batch_bucket(const SetView* sv, const int32_t* offs, int nsets, int64_t total, cudaStream_t st) {
    if (total < 1) return cudaSuccess;
    k_batch_count<<<nb(total), 256, 0, st>>>(sv, offs, nsets);
    k_batch_scan<<<nsets, SCAN_THREADS, 0, st>>>(sv);
    k_batch_scatter<<<nb(total), 256, 0, st>>>(sv, offs, nsets);
    k_batch_rank<<<nb(total), 256, 0, st>>>(sv, offs, nsets);
    return cudaGetLastError();
}

cudaError_t launch_batch_move(const SetView* sv, const int32_t* offs, int nsets, int64_t total, css_integrator it,
                              int half, int* status, cudaStream_t st) {
    if (total < 1) return cudaSuccess;
    if (it.kind == CSS_INT_NVE) {
        if (half == 0) k_batch_kick_drift<<<nb(total, 128), 128, 0, st>>>(sv, offs, nsets, it, status);
        else k_batch_kick<<<nb(total), 256, 0, st>>>(sv, offs, nsets, 0.5 * it.dt / it.mass);
    } else if (half == 1) {
        k_batch_overdamped<<<nb(total, 128), 128, 0, st>>>(sv, offs, nsets, it, status);
        k_batch_step_inc<<<nb(nsets), 256, 0, st>>>(sv, nsets);
    }
    return cudaGetLastError();
}


}  // namespace cssi
