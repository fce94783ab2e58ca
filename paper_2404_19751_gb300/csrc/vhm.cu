// vhm.cu -- approximate geodesic distances and initial tangents: heat-method distances
// with vector-heat transport, the approximate alternative to exact window propagation
// that the paper names (Sec. 2.2: the vector heat method with O(h) distance error on a
// mesh of spacing h; Sec. 5: other solvers as future work).
//
// For a source q (face f0, barycentrics b), with t = t_factor * h^2 (h: mean edge length):
//   (M + t L) u = u0         scalar heat, one backward-Euler step, u0 = b on f0's corners
//   (M + t Lc) Y = Y0        vector heat, Y0 = b_k times f0's layout x-axis in corner k's frame
//   X = -grad u / |grad u|   per face (0 where the gradient vanishes)
//   L phi = -div X           Poisson, right-hand side made mean-free; phi(q) = 0
// and for a target y in face g (barycentrics c): d = phi(y) (linear interpolation); the
// tangent at q is f0's x-axis turned by arg sum_k c_k exp(i psi_k) conj(H_k), psi_k the
// angle of grad phi on g in corner k's frame and H = Y / |Y| the transported reference.
// L is the cotan Laplacian (w_ij = (cot a + cot b) / 2), M the lumped mass, Lc the
// connection Laplacian over vertex frames whose corner angles are scaled by
// s_v = 2 pi / Theta_v (pi / Theta_v on the boundary) so that they close up; a vector at
// neighbour j enters vertex i's frame turned by phi_ij + pi - phi_ji (phi_ij: the angle
// at i of the edge towards j).
//
// GPU organisation: K sources at a time (K a power of two <= 256), fields vertex-major
// with the K sources contiguous, thread (v, s) at v K + s, so the K threads of a row share
// the row's operator entries.  The heat systems are solved by Gauss-Seidel sweeps over a
// colouring of the vertex graph (one launch per colour): the matrices are symmetric positive
// definite, so the sweeps converge on any mesh; where the scalar matrix is an M-matrix every
// sweep adds non-negative terms, and the solution keeps its relative accuracy where it is
// tiny far from the source (a Krylov solver's residual norm would not); the sweeps stop when
// no entry changes by more than 1e-14 of the terms it is summed from.  The
// Poisson system is solved by Jacobi-preconditioned conjugate gradients, one column per
// source, with per-source reductions in a fixed order (the result does not depend on
// thread timing).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "css_internal.h"

namespace {

constexpr double VPI = 3.141592653589793238462643383279503;
constexpr int VT = 256;   // threads per block of the (vertex, source) kernels

inline unsigned vblk(int64_t n, int b = VT) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ double wrap_pi(double a) {   // into (-pi, pi]
    return a - 2.0 * VPI * ceil((a - VPI) / (2.0 * VPI));
}

// corner k of face f in its layout: corner 0 at the origin, corner 1 on +x, corner 2 above
__device__ __forceinline__ void lay_corner(const double* lay, int f, int k, double& x, double& y) {
    if (k == 0) { x = 0.0; y = 0.0; }
    else if (k == 1) { x = lay[3 * f]; y = 0.0; }
    else { x = lay[3 * f + 1]; y = lay[3 * f + 2]; }
}

// ------------------------------------------------------------------ operators (once per mesh)
// per corner: angle, its cotangent, the layout angle of the outgoing edge; per face: area
__global__ void k_corners(int32_t nf, const double* lay, double* ang, double* cot, double* gam, double* area) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    double px[3], py[3];
    for (int k = 0; k < 3; ++k) lay_corner(lay, f, k, px[k], py[k]);
    for (int k = 0; k < 3; ++k) {
        const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
        const double ux = px[k1] - px[k], uy = py[k1] - py[k], wx = px[k2] - px[k], wy = py[k2] - py[k];
        const double a = atan2(ux * wy - uy * wx, ux * wx + uy * wy);
        ang[3 * f + k] = a;
        cot[3 * f + k] = cos(a) / sin(a);
        gam[3 * f + k] = atan2(uy, ux);
    }
    area[f] = 0.5 * lay[3 * f] * lay[3 * f + 2];
}

// per vertex: mass, frame scale, the frame angle of each corner (walked counter-clockwise
// from the vertex's reference corner) and each corner's position in the ring
__global__ void k_frames(int32_t nv, const int32_t* ring_start, const int32_t* ring, const int32_t* twin,
                         const uint8_t* bnd, const double* theta, const double* ang, const double* area, double* mass,
                         double* scale, double* phi, int32_t* pos, int* status) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int s = ring_start[v], e = ring_start[v + 1], deg = e - s;
    double m = 0.0;
    for (int p = s; p < e; ++p) {
        const int h = ring[p];
        m += area[h / 3] / 3.0;
        pos[h] = p;
    }
    mass[v] = m;
    const double sc = (bnd[v] ? VPI : 2.0 * VPI) / theta[v];
    scale[v] = sc;
    int start = ring[s];   // the ring is sorted: the smallest corner id
    if (bnd[v]) {          // a boundary fan starts at the corner whose outgoing edge has no twin
        for (int p = s; p < e; ++p)
            if (twin[ring[p]] < 0) { start = ring[p]; break; }
    }
    int h = start, seen = 0;
    double acc = 0.0;
    while (seen < deg) {
        phi[h] = sc * acc;
        acc += ang[h];
        ++seen;
        const int f = h / 3, k = h - 3 * f;
        const int nxt = twin[3 * f + (k == 0 ? 2 : k - 1)];   // across the corner's incoming edge
        if (nxt < 0 || nxt == start) break;
        h = nxt;
    }
    if (seen != deg) atomicOr(status, 1);   // not a single disk or half-disk around v
}

// two row entries per corner (the two edges of the corner's face at its vertex): neighbour,
// half cotan weight of the face's corner opposite the edge, and the turn that carries a
// vector at the neighbour into the row vertex's frame
__global__ void k_entries(int32_t nf, const int32_t* fv, const double* ang, const double* cot, const double* phi,
                          const double* scale, const int32_t* pos, int32_t* ej, double* ew, double* ec, double* es) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * nf) return;
    const int f = h / 3, k = h - 3 * f;
    const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
    const int v = fv[h], j1 = fv[3 * f + k1], j2 = fv[3 * f + k2];
    const int o = 2 * pos[h];
    // edge v -> j1 (the corner's outgoing edge); j1 sees the edge j1 -> v turned by its corner
    // angle from its own outgoing edge
    const double a1 = phi[h] + VPI - (phi[3 * f + k1] + scale[j1] * ang[3 * f + k1]);
    ej[o] = j1;
    ew[o] = 0.5 * cot[3 * f + k2];
    ec[o] = cos(a1);
    es[o] = sin(a1);
    // edge v -> j2, turned by v's corner angle from v's outgoing edge; at j2 it is j2's
    // outgoing edge in this face
    const double a2 = phi[h] + scale[v] * ang[h] + VPI - phi[3 * f + k2];
    ej[o + 1] = j2;
    ew[o + 1] = 0.5 * cot[3 * f + k1];
    ec[o + 1] = cos(a2);
    es[o + 1] = sin(a2);
}

__global__ void k_rowsum(int32_t nv, const int32_t* ring_start, const double* ew, double* diag) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double s = 0.0;
    for (int e = 2 * ring_start[v]; e < 2 * ring_start[v + 1]; ++e) s += ew[e];
    diag[v] = s;
}

// mean of the three side lengths of every face, in a fixed order (one block)
__global__ void k_mean_edge(int32_t nf, const double* lay, double* out) {
    __shared__ double sh[1024];
    double s = 0.0;
    for (int f = threadIdx.x; f < nf; f += blockDim.x) {
        const double L01 = lay[3 * f], x2 = lay[3 * f + 1], y2 = lay[3 * f + 2];
        s += L01 + sqrt(x2 * x2 + y2 * y2) + sqrt((x2 - L01) * (x2 - L01) + y2 * y2);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / (3.0 * nf);
}

// ------------------------------------------------------------------ per-batch solves
struct Op {
    int32_t nv, nf;
    const int32_t* fv;
    const double* lay;
    const double* frame;
    const int32_t* ring_start;
    const int32_t* ring;
    const double* mass;
    const double* diag;
    const double* scale;
    const double* phi;
    const double* gam;
    const double* cot;
    const int32_t* ej;
    const double* ew;
    const double* ec;
    const double* es;
};

// right-hand sides of both heat steps for source column s (K columns; inactive columns: 0)
__global__ void k_heat_rhs(Op o, int K, int nsrc, const int32_t* src, const int32_t* face, const double* bary,
                           double* bu, double* bY) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nsrc) return;
    const int s = t / 3, k = t - 3 * s;
    const int i = src[s], f0 = face[i];
    const int v = o.fv[3 * f0 + k];
    const double b = bary[3 * (size_t)i + k];
    const double psi = o.phi[3 * f0 + k] + o.scale[v] * wrap_pi(0.0 - o.gam[3 * f0 + k]);
    const size_t a = (size_t)v * K + s;
    bu[a] = b;   // the three corners of a face are distinct vertices
    bY[2 * a] = b * cos(psi);
    bY[2 * a + 1] = b * sin(psi);
}

// per call: the heat step's entries scaled by t (weight, and weight times the transport turn)
// and the inverse diagonal, so a sweep spends five FP64 operations per entry
__global__ void k_heat_entries(Op o, double t, double* wt, double* wc, double* wsn, double* inv_d) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < 6 * o.nf) {
        const double w = t * o.ew[e];
        wt[e] = w;
        wc[e] = w * o.ec[e];
        wsn[e] = w * o.es[e];
    }
    if (e < o.nv) inv_d[e] = 1.0 / (o.mass[e] + t * o.diag[e]);
}

// One colour of a Gauss-Seidel sweep of both heat systems, in place: every vertex of the
// colour takes x_v <- D_v^-1 (b_v + t sum_j w_vj x_j) from its neighbours' current values (no
// two vertices of a colour are neighbours, so the order within a colour does not matter).
// (M + t L) is symmetric positive definite for any mesh (L is the Dirichlet form of the
// piecewise-linear interpolant, the connection Laplacian that of the transported field), so
// the sweeps converge without damping; with all weights positive every term is
// non-negative, which keeps far-field entries relatively accurate.  With check, entries
// that still change by more than 1e-14 of the magnitude of the terms they are summed from
// raise *flag (an entry the sweeps have not reached is 0 and changes when they do, so the
// flag stays up until every vertex has been reached; below 1e-290 an entry has no relative
// accuracy left to converge to).
__global__ void __launch_bounds__(VT) k_heat_gs(Op o, int K, int nsrc, const double* wt, const double* wc,
                                                const double* wsn, const double* inv_d, const int32_t* verts,
                                                int nverts, const double* bu, const double* bY, double* u, double* Y,
                                                int check, int* flag) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool moved = false;
    const int s = (int)(g % K);
    if (g < (int64_t)nverts * K && s < nsrc) {   // columns beyond the batch's sources stay 0
        const int v = verts[g / K];
        const size_t a = (size_t)v * K + s;
        double au = bu[a], ar = bY[2 * a], ai = bY[2 * a + 1];
        double su = 0.0, sy = 0.0;   // magnitudes of the summed terms (for the check only)
        for (int e = 2 * o.ring_start[v]; e < 2 * o.ring_start[v + 1]; ++e) {
            const size_t j = (size_t)o.ej[e] * K + s;
            const double w = wt[e], c = wc[e], sn = wsn[e];
            const double uj = u[j], yr = Y[2 * j], yi = Y[2 * j + 1];
            au += w * uj;
            ar += c * yr - sn * yi;
            ai += sn * yr + c * yi;
            if (check) {
                su += fabs(w * uj);
                sy += fabs(w) * sqrt(yr * yr + yi * yi);
            }
        }
        if (check) {
            su += fabs(bu[a]);
            sy += sqrt(bY[2 * a] * bY[2 * a] + bY[2 * a + 1] * bY[2 * a + 1]);
        }
        const double iD = inv_d[v];
        const double nu = au * iD, nr = ar * iD, ni = ai * iD;
        if (check) {
            const double su_d = su * iD, sy_d = sy * iD;
            const double dr = nr - Y[2 * a], di = ni - Y[2 * a + 1];
            moved = (su_d > 1e-290 && fabs(nu - u[a]) > 1e-14 * su_d) ||
                    (sy_d > 1e-290 && sqrt(dr * dr + di * di) > 1e-14 * sy_d);
        }
        u[a] = nu;
        Y[2 * a] = nr;
        Y[2 * a + 1] = ni;
    }
    if (check && __any_sync(CSS_FULL, moved) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// X = -grad u / |grad u| per (face, column)
__global__ void k_unit_field(Op o, int K, const double* u, double* X) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)o.nf * K) return;
    const int f = (int)(g / K), s = (int)(g - (int64_t)f * K);
    double px[3], py[3];
    for (int k = 0; k < 3; ++k) lay_corner(o.lay, f, k, px[k], py[k]);
    const double A2 = o.lay[3 * f] * o.lay[3 * f + 2];   // twice the area
    double gx = 0.0, gy = 0.0;
    for (int k = 0; k < 3; ++k) {
        const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
        const double ex = px[k2] - px[k1], ey = py[k2] - py[k1];
        const double uk = u[(size_t)o.fv[3 * f + k] * K + s];
        gx += uk * -ey;
        gy += uk * ex;
    }
    gx /= A2;
    gy /= A2;
    const double n = sqrt(gx * gx + gy * gy);
    X[2 * g] = n > 0.0 ? -gx / n : 0.0;
    X[2 * g + 1] = n > 0.0 ? -gy / n : 0.0;
}

// Poisson right-hand side -div X per (vertex, column); inactive columns get 0
__global__ void k_neg_div(Op o, int K, int nsrc, const double* X, double* b) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)o.nv * K) return;
    const int v = (int)(g / K), s = (int)(g - (int64_t)v * K);
    double acc = 0.0;
    if (s < nsrc) {
        for (int p = o.ring_start[v]; p < o.ring_start[v + 1]; ++p) {
            const int h = o.ring[p], f = h / 3, k = h - 3 * f;
            const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
            double x0, y0, x1, y1, x2, y2;
            lay_corner(o.lay, f, k, x0, y0);
            lay_corner(o.lay, f, k1, x1, y1);
            lay_corner(o.lay, f, k2, x2, y2);
            const double Xx = X[2 * ((size_t)f * K + s)], Xy = X[2 * ((size_t)f * K + s) + 1];
            acc += 0.5 * (o.cot[3 * f + k2] * ((x1 - x0) * Xx + (y1 - y0) * Xy) +
                          o.cot[3 * f + k1] * ((x2 - x0) * Xx + (y2 - y0) * Xy));
        }
    }
    b[g] = -acc;
}

// Per-block partial sums of a (vertex, column) product, per column: block b covers the
// rows [b VT / K, (b + 1) VT / K) (K divides VT), and thread s < K sums its column over
// them in row order.
__device__ __forceinline__ void block_partial(double val, int K, double* partial) {
    __shared__ double sh[VT];
    sh[threadIdx.x] = val;
    __syncthreads();
    if ((int)threadIdx.x < K) {
        double s = 0.0;
        for (int r = 0; r < VT / K; ++r) s += sh[r * K + threadIdx.x];
        partial[(size_t)blockIdx.x * K + threadIdx.x] = s;
    }
}

// per column: the sum of its nb block partials in a fixed order (one block per column)
__global__ void k_col_sum(int K, int nb, const double* partial, double* out) {
    __shared__ double sh[VT];
    const int s = blockIdx.x;
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) a += partial[(size_t)b * K + s];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[s] = sh[0];
}

__global__ void k_partial_of(Op o, int K, const double* x, double* partial) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    block_partial(g < (int64_t)o.nv * K ? x[g] : 0.0, K, partial);
}

// b -= mean(b) per column; CG start: x = 0, r = b, z = r / diag, p = z, partial r.z
__global__ void k_cg_start(Op o, int K, const double* bsum, double* b, double* x, double* r, double* z, double* p,
                           double* partial) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double rz = 0.0;
    if (g < (int64_t)o.nv * K) {
        const int v = (int)(g / K), s = (int)(g - (int64_t)v * K);
        const double bb = b[g] - bsum[s] / o.nv;
        b[g] = bb;
        x[g] = 0.0;
        r[g] = bb;
        const double zz = bb / o.diag[v];
        z[g] = zz;
        p[g] = zz;
        rz = bb * zz;
    }
    block_partial(rz, K, partial);
}

// q = L p, partial p.q
__global__ void k_cg_apply(Op o, int K, const double* p, double* q, double* partial) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double pq = 0.0;
    if (g < (int64_t)o.nv * K) {
        const int v = (int)(g / K), s = (int)(g - (int64_t)v * K);
        double a = o.diag[v] * p[g];
        for (int e = 2 * o.ring_start[v]; e < 2 * o.ring_start[v + 1]; ++e) a -= o.ew[e] * p[(size_t)o.ej[e] * K + s];
        q[g] = a;
        pq = p[g] * a;
    }
    block_partial(pq, K, partial);
}

// per column: alpha = rz / pq while active (0 once converged)
__global__ void k_cg_alpha(int K, const double* rz, const double* pq, const int* active, double* alpha) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < K) alpha[s] = (active[s] && pq[s] != 0.0) ? rz[s] / pq[s] : 0.0;
}

// x += alpha p, r -= alpha q, z = r / diag, partial r.z
__global__ void k_cg_step(Op o, int K, const double* alpha, const double* p, const double* q, double* x, double* r,
                          double* z, double* partial) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double rz = 0.0;
    if (g < (int64_t)o.nv * K) {
        const int v = (int)(g / K), s = (int)(g - (int64_t)v * K);
        const double a = alpha[s];
        x[g] += a * p[g];
        const double rr = r[g] - a * q[g];
        r[g] = rr;
        const double zz = rr / o.diag[v];
        z[g] = zz;
        rz = rr * zz;
    }
    block_partial(rz, K, partial);
}

// per column: beta = rz_new / rz, convergence (rz <= tol^2 rz0), counts the active ones
__global__ void k_cg_beta(int K, double tol2, const double* rz0, double* rz, const double* rzn, int* active,
                          double* beta, int* n_active) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= K) return;
    if (!active[s]) { beta[s] = 0.0; return; }
    beta[s] = rz[s] != 0.0 ? rzn[s] / rz[s] : 0.0;
    rz[s] = rzn[s];
    if (!(rzn[s] > tol2 * rz0[s])) active[s] = 0;
    else atomicAdd(n_active, 1);
}

// p = z + beta p on the columns still active
__global__ void k_cg_dir(Op o, int K, const int* active, const double* beta, const double* z, double* p) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)o.nv * K) return;
    const int s = (int)(g % K);
    if (active[s]) p[g] = z[g] + beta[s] * p[g];
}

// distance and world tangent of target j from source column s; keep = (j != i, d < r_c)
__global__ void k_evaluate(Op o, int K, int nsrc, int n, const int32_t* src, const int32_t* face, const double* bary,
                           const double* phi, const double* Y, double rc, double* od, double* ot, int32_t* keep) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)nsrc * n) return;
    const int s = (int)(g / n), j = (int)(g - (int64_t)s * n);
    const int i = src[s], f0 = face[i], fg = face[j];
    const double* c = bary + 3 * (size_t)j;
    double ph[3];
    int vk[3];
    for (int k = 0; k < 3; ++k) {
        vk[k] = o.fv[3 * fg + k];
        ph[k] = phi[(size_t)vk[k] * K + s];
    }
    // phi at the source point (the gauge phi(q) = 0)
    double p0 = 0.0;
    for (int k = 0; k < 3; ++k) p0 += bary[3 * (size_t)i + k] * phi[(size_t)o.fv[3 * f0 + k] * K + s];
    const double d = c[0] * ph[0] + c[1] * ph[1] + c[2] * ph[2] - p0;
    // grad phi on the target's face, its angle in each corner's frame against the transported
    // reference there
    double px[3], py[3];
    for (int k = 0; k < 3; ++k) lay_corner(o.lay, fg, k, px[k], py[k]);
    const double A2 = o.lay[3 * fg] * o.lay[3 * fg + 2];
    double gx = 0.0, gy = 0.0;
    for (int k = 0; k < 3; ++k) {
        const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
        gx += ph[k] * -(py[k2] - py[k1]);
        gy += ph[k] * (px[k2] - px[k1]);
    }
    gx /= A2;
    gy /= A2;
    const double beta = atan2(gy, gx);
    double zr = 0.0, zi = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double psi = o.phi[3 * fg + k] + o.scale[vk[k]] * wrap_pi(beta - o.gam[3 * fg + k]);
        const double yr = Y[2 * ((size_t)vk[k] * K + s)], yi = Y[2 * ((size_t)vk[k] * K + s) + 1];
        const double yn = sqrt(yr * yr + yi * yi);
        if (!(yn > 0.0)) continue;
        const double hr = yr / yn, hi = yi / yn;
        const double er = cos(psi), ei = sin(psi);
        zr += c[k] * (er * hr + ei * hi);   // exp(i psi) conj(H)
        zi += c[k] * (ei * hr - er * hi);
    }
    const double th = atan2(zi, zr);
    const double ct = cos(th), st = sin(th);
    const double* fr = o.frame + 9 * (size_t)f0;
    od[g] = d;
    ot[3 * g] = ct * fr[3] + st * fr[6];
    ot[3 * g + 1] = ct * fr[4] + st * fr[7];
    ot[3 * g + 2] = ct * fr[5] + st * fr[8];
    keep[g] = (j != i && d < rc) ? 1 : 0;
}

// per source column: its kept pairs in increasing j, written at base + the running count
// (one block per column, a block-wide scan over j in chunks)
__global__ void k_compact_rows(int n, const int32_t* keep, const double* od, const double* ot,
                               const int64_t* row_off, int32_t* oj, double* odist, double* otan) {
    __shared__ int sh[VT];
    const int s = blockIdx.x;
    int64_t base = row_off[s];
    for (int j0 = 0; j0 < n; j0 += VT) {
        const int j = j0 + threadIdx.x;
        const size_t g = (size_t)s * n + j;
        const int k = j < n ? keep[g] : 0;
        sh[threadIdx.x] = k;
        __syncthreads();
        for (int w = 1; w < VT; w <<= 1) {   // inclusive scan
            const int add = (int)threadIdx.x >= w ? sh[threadIdx.x - w] : 0;
            __syncthreads();
            sh[threadIdx.x] += add;
            __syncthreads();
        }
        if (k) {
            const int64_t o = base + sh[threadIdx.x] - 1;
            oj[o] = j;
            odist[o] = od[g];
            otan[3 * o] = ot[3 * g];
            otan[3 * o + 1] = ot[3 * g + 1];
            otan[3 * o + 2] = ot[3 * g + 2];
        }
        base += sh[VT - 1];
        __syncthreads();
    }
}

__global__ void k_count_rows(int n, const int32_t* keep, int64_t* cnt) {
    __shared__ int sh[VT];
    const int s = blockIdx.x;
    int a = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) a += keep[(size_t)s * n + j];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) cnt[s] = sh[0];
}

}  // namespace

// ===================================================================================== host
namespace cssi {

struct VhmOp {
    int32_t nv = 0, nf = 0;
    double h = 0.0;   // mean edge length
    double *ang = nullptr, *cot = nullptr, *gam = nullptr, *area = nullptr, *mass = nullptr, *diag = nullptr,
           *scale = nullptr, *phi = nullptr, *ew = nullptr, *ec = nullptr, *es = nullptr;
    int32_t *pos = nullptr, *ej = nullptr;
    int32_t* cverts = nullptr;        // vertices grouped by colour (no two neighbours share one)
    std::vector<int32_t> cstart;      // colour c is cverts[cstart[c] .. cstart[c + 1])
};

void vhm_free(css_mesh* m) {
    VhmOp* o = m->vhm;
    if (!o) return;
    cudaFree(o->ang); cudaFree(o->cot); cudaFree(o->gam); cudaFree(o->area); cudaFree(o->mass);
    cudaFree(o->diag); cudaFree(o->scale); cudaFree(o->phi); cudaFree(o->ew); cudaFree(o->ec); cudaFree(o->es);
    cudaFree(o->pos); cudaFree(o->ej); cudaFree(o->cverts);
    delete o;
    m->vhm = nullptr;
}

}  // namespace cssi

namespace {

#define VTRY(what, x)                                                                            \
    do {                                                                                         \
        cudaError_t e__ = (x);                                                                   \
        if (e__ != cudaSuccess) {                                                                \
            c->err = std::string(what) + ": " + cudaGetErrorString(e__);                         \
            return e__ == cudaErrorMemoryAllocation ? CSS_ERR_OOM : CSS_ERR_CUDA;                \
        }                                                                                        \
    } while (0)

int build_op(css_mesh* m) {
    css_ctx* c = m->ctx;
    if (m->vhm) return CSS_OK;
    cssi::VhmOp* o = new cssi::VhmOp();
    m->vhm = o;
    const int32_t nv = (int32_t)m->nv, nf = (int32_t)m->nf;
    o->nv = nv;
    o->nf = nf;
    cudaStream_t st = c->stream;
    VTRY("vhm operators", cudaMalloc(&o->ang, 3 * (size_t)nf * sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&o->cot, 3 * (size_t)nf * sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&o->gam, 3 * (size_t)nf * sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&o->phi, 3 * (size_t)nf * sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&o->pos, 3 * (size_t)nf * sizeof(int32_t)));
    VTRY("vhm operators", cudaMalloc(&o->area, (size_t)nf * sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&o->mass, (size_t)nv * sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&o->diag, (size_t)nv * sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&o->scale, (size_t)nv * sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&o->ej, 6 * (size_t)nf * sizeof(int32_t)));
    VTRY("vhm operators", cudaMalloc(&o->ew, 6 * (size_t)nf * sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&o->ec, 6 * (size_t)nf * sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&o->es, 6 * (size_t)nf * sizeof(double)));
    double* dh = nullptr;
    int* dst = nullptr;
    VTRY("vhm operators", cudaMalloc(&dh, sizeof(double)));
    VTRY("vhm operators", cudaMalloc(&dst, sizeof(int)));
    cudaError_t e = cudaMemsetAsync(dst, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        k_corners<<<vblk(nf), VT, 0, st>>>(nf, m->lay, o->ang, o->cot, o->gam, o->area);
        k_frames<<<vblk(nv), VT, 0, st>>>(nv, m->ring_start, m->ring, m->twin, m->bnd, m->theta, o->ang, o->area,
                                          o->mass, o->scale, o->phi, o->pos, dst);
        k_entries<<<vblk(3 * (int64_t)nf), VT, 0, st>>>(nf, m->fv, o->ang, o->cot, o->phi, o->scale, o->pos, o->ej,
                                                         o->ew, o->ec, o->es);
        k_rowsum<<<vblk(nv), VT, 0, st>>>(nv, m->ring_start, o->ew, o->diag);
        k_mean_edge<<<1, 1024, 0, st>>>(nf, m->lay, dh);
        e = cudaGetLastError();
    }
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&o->h, dh, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, dst, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dh);
    cudaFree(dst);
    if (e != cudaSuccess) {
        cssi::vhm_free(m);
        c->err = std::string("vhm operators: ") + cudaGetErrorString(e);
        return CSS_ERR_CUDA;
    }
    if (status) {
        cssi::vhm_free(m);
        c->err = "vhm: a vertex's faces do not form one disk or half-disk";
        return CSS_ERR_NONMANIFOLD;
    }
    // greedy colouring of the vertex graph (each vertex takes the smallest colour none of its
    // already coloured neighbours has), for the Gauss-Seidel sweeps
    std::vector<int32_t> rs((size_t)nv + 1), ej((size_t)6 * nf);
    e = cudaMemcpyAsync(rs.data(), m->ring_start, rs.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ej.data(), o->ej, ej.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cssi::vhm_free(m);
        c->err = std::string("vhm operators: ") + cudaGetErrorString(e);
        return CSS_ERR_CUDA;
    }
    std::vector<int32_t> col((size_t)nv, -1);
    std::vector<char> used;
    int ncol = 0;
    for (int32_t v = 0; v < nv; ++v) {
        used.assign((size_t)ncol + 1, 0);
        for (int32_t k = 2 * rs[v]; k < 2 * rs[v + 1]; ++k) {
            const int32_t j = ej[k];
            if (j != v && col[j] >= 0) used[col[j]] = 1;
        }
        int cv = 0;
        while (used[cv]) ++cv;
        col[v] = cv;
        ncol = std::max(ncol, cv + 1);
    }
    o->cstart.assign((size_t)ncol + 1, 0);
    for (int32_t v = 0; v < nv; ++v) ++o->cstart[col[v] + 1];
    for (int cc = 0; cc < ncol; ++cc) o->cstart[cc + 1] += o->cstart[cc];
    std::vector<int32_t> order((size_t)nv), fill(o->cstart.begin(), o->cstart.end() - 1);
    for (int32_t v = 0; v < nv; ++v) order[fill[col[v]]++] = v;
    e = cudaMalloc(&o->cverts, std::max<size_t>(nv, 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemcpyAsync(o->cverts, order.data(), (size_t)nv * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cssi::vhm_free(m);
        c->err = std::string("vhm operators: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? CSS_ERR_OOM : CSS_ERR_CUDA;
    }
    return CSS_OK;
}

bool dev_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// an executable graph, destroyed with its owner
struct GraphExec {
    cudaGraphExec_t exec = nullptr;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
    ~GraphExec() { reset(); }
};

// device buffers of one batch of K columns
struct Batch {
    std::vector<void*> owned;
    double *u = nullptr, *Y = nullptr, *bu = nullptr, *bY = nullptr, *X = nullptr,
           *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *partial = nullptr,
           *sc = nullptr, *od = nullptr, *ot = nullptr, *pj_d = nullptr, *pj_t = nullptr, *wt = nullptr, *wc = nullptr,
           *wsn = nullptr, *invd = nullptr;
    int32_t *src = nullptr, *keep = nullptr, *pj = nullptr;
    int* ints = nullptr;   // [0] flag, [1] active count, [2..2+K) active
    int64_t* cnt = nullptr;
    int64_t* roff = nullptr;
    ~Batch() { for (void* a : owned) cudaFree(a); }
    template <class T>
    cudaError_t get(T** out, size_t n) {
        void* a = nullptr;
        cudaError_t e = cudaMalloc(&a, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) owned.push_back(a);
        *out = (T*)a;
        return e;
    }
};

}  // namespace

int css_vhm_neighbors(css_parts* parts, double r_c, double t_factor, int64_t capacity, int64_t* n_pairs,
                      int64_t* row_start, int32_t* nbr_j, double* dist, double* tangent) {
    if (!parts || !n_pairs || !(r_c > 0.0) || !(t_factor > 0.0) || !std::isfinite(t_factor) || capacity < 0)
        return CSS_ERR_INVALID_ARG;
    css_ctx* c = parts->ctx;
    css_mesh* m = parts->mesh;
    int rc = build_op(m);
    if (rc) return rc;
    const cssi::VhmOp& O = *m->vhm;
    cudaStream_t st = c->stream;
    const int32_t n = (int32_t)parts->n, nv = O.nv, nf = O.nf;
    const double t = t_factor * O.h * O.h;
    // columns per batch: a power of two <= 256 that keeps the batch's fields near 2 GB
    int K = 256;
    while (K > 1 && ((double)K * (18.0 * nv + 2.0 * nf) * 8.0 + (double)K * n * 40.0 > 2.0e9 || K / 2 >= n)) K /= 2;
    Op op{nv, nf, m->fv, m->lay, m->frame, m->ring_start, m->ring, O.mass, O.diag, O.scale, O.phi, O.gam, O.cot,
          O.ej, O.ew, O.ec, O.es};
    Batch B;
    const size_t VK = (size_t)nv * K;
    const int nbv = (int)vblk((int64_t)VK);
    VTRY("vhm", B.get(&B.u, VK)); VTRY("vhm", B.get(&B.Y, 2 * VK));
    VTRY("vhm", B.get(&B.bu, VK)); VTRY("vhm", B.get(&B.bY, 2 * VK));
    VTRY("vhm", B.get(&B.X, 2 * (size_t)nf * K)); VTRY("vhm", B.get(&B.b, VK)); VTRY("vhm", B.get(&B.x, VK));
    VTRY("vhm", B.get(&B.r, VK)); VTRY("vhm", B.get(&B.z, VK)); VTRY("vhm", B.get(&B.p, VK));
    VTRY("vhm", B.get(&B.q, VK)); VTRY("vhm", B.get(&B.partial, (size_t)nbv * K));
    VTRY("vhm", B.get(&B.sc, 8 * (size_t)K)); VTRY("vhm", B.get(&B.src, (size_t)K));
    VTRY("vhm", B.get(&B.ints, 2 + (size_t)K)); VTRY("vhm", B.get(&B.cnt, (size_t)K));
    VTRY("vhm", B.get(&B.roff, (size_t)K));
    VTRY("vhm", B.get(&B.od, (size_t)K * n)); VTRY("vhm", B.get(&B.ot, 3 * (size_t)K * n));
    VTRY("vhm", B.get(&B.keep, (size_t)K * n));
    VTRY("vhm", B.get(&B.wt, 6 * (size_t)nf)); VTRY("vhm", B.get(&B.wc, 6 * (size_t)nf));
    VTRY("vhm", B.get(&B.wsn, 6 * (size_t)nf)); VTRY("vhm", B.get(&B.invd, (size_t)nv));
    k_heat_entries<<<vblk(std::max<int64_t>(6 * (int64_t)nf, nv)), VT, 0, st>>>(op, t, B.wt, B.wc, B.wsn, B.invd);
    VTRY("vhm", cudaGetLastError());
    double* bsum = B.sc;          // K
    double* rz = B.sc + K;        // K
    double* rz0 = B.sc + 2 * K;   // K
    double* pq = B.sc + 3 * K;    // K
    double* rzn = B.sc + 4 * K;   // K
    double* alpha = B.sc + 5 * K; // K
    double* beta = B.sc + 6 * K;  // K
    int* flag = B.ints;
    int* nact = B.ints + 1;
    int* active = B.ints + 2;
    // outputs: device pointers are written in place, host ones through a staging copy per batch
    const bool dev_out = dev_ptr(nbr_j) && dev_ptr(dist) && dev_ptr(tangent);
    std::vector<int64_t> rows((size_t)n + 1, 0);
    int64_t total = 0;
    int64_t iters_heat = 0, iters_cg = 0;
    const int MAX_SWEEPS = 50000, MAX_CG = 50000, CHUNK = 16;
    GraphExec chunk;
    int chunk_ns = -1;
    for (int s0 = 0; s0 < n; s0 += K) {
        const int ns = std::min(K, n - s0);
        std::vector<int32_t> hsrc(K);
        for (int s = 0; s < K; ++s) hsrc[s] = s0 + std::min(s, ns - 1);
        VTRY("vhm", cudaMemcpyAsync(B.src, hsrc.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        // ---- heat steps (Gauss-Seidel sweeps from zero, colour by colour)
        VTRY("vhm", cudaMemsetAsync(B.bu, 0, VK * sizeof(double), st));
        VTRY("vhm", cudaMemsetAsync(B.bY, 0, 2 * VK * sizeof(double), st));
        VTRY("vhm", cudaMemsetAsync(B.u, 0, VK * sizeof(double), st));
        VTRY("vhm", cudaMemsetAsync(B.Y, 0, 2 * VK * sizeof(double), st));
        k_heat_rhs<<<vblk(3 * ns), VT, 0, st>>>(op, K, ns, B.src, parts->face, parts->bary, B.bu, B.bY);
        VTRY("vhm heat", cudaGetLastError());
        double *u = B.u, *Y = B.Y;
        int sweeps = 0;
        // a chunk of sweeps (one launch per colour and sweep) is captured once as a graph and
        // replayed: on small meshes the launches, not the sweeps, would set the time
        if (!chunk.exec || chunk_ns != ns) {
            chunk.reset();
            cudaGraph_t graph = nullptr;
            VTRY("vhm capture", cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
            const int ncol = (int)O.cstart.size() - 1;
            for (int k = 0; k < CHUNK && e == cudaSuccess; ++k)
                for (int cc = 0; cc < ncol; ++cc) {
                    const int nvc = O.cstart[cc + 1] - O.cstart[cc];
                    k_heat_gs<<<vblk((int64_t)nvc * K), VT, 0, st>>>(op, K, ns, B.wt, B.wc, B.wsn, B.invd,
                                                                      O.cverts + O.cstart[cc], nvc, B.bu, B.bY, u, Y,
                                                                      k == CHUNK - 1, flag);
                }
            if (e == cudaSuccess) e = cudaGetLastError();
            const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&chunk.exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            VTRY("vhm capture", e);
            chunk_ns = ns;
        }
        for (;;) {
            VTRY("vhm heat", cudaGraphLaunch(chunk.exec, st));
            sweeps += CHUNK;
            int hf = 0;
            VTRY("vhm heat", cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
            VTRY("vhm heat", cudaStreamSynchronize(st));
            if (!hf) break;
            if (sweeps >= MAX_SWEEPS) { c->err = "vhm: heat sweeps did not converge"; return CSS_ERR_ITER_LIMIT; }
        }
        iters_heat = std::max<int64_t>(iters_heat, sweeps);
        // ---- unit field, Poisson right-hand side (mean-free), conjugate gradients
        const int nbf = (int)vblk((int64_t)nf * K);
        k_unit_field<<<nbf, VT, 0, st>>>(op, K, u, B.X);
        k_neg_div<<<nbv, VT, 0, st>>>(op, K, ns, B.X, B.b);
        k_partial_of<<<nbv, VT, 0, st>>>(op, K, B.b, B.partial);
        k_col_sum<<<K, VT, 0, st>>>(K, nbv, B.partial, bsum);
        k_cg_start<<<nbv, VT, 0, st>>>(op, K, bsum, B.b, B.x, B.r, B.z, B.p, B.partial);
        k_col_sum<<<K, VT, 0, st>>>(K, nbv, B.partial, rz);
        VTRY("vhm poisson", cudaGetLastError());
        VTRY("vhm poisson", cudaMemcpyAsync(rz0, rz, K * sizeof(double), cudaMemcpyDeviceToDevice, st));
        {
            std::vector<int> ha(K);
            for (int s = 0; s < K; ++s) ha[s] = s < ns ? 1 : 0;
            VTRY("vhm poisson", cudaMemcpyAsync(active, ha.data(), K * sizeof(int), cudaMemcpyHostToDevice, st));
        }
        int cg = 0;
        for (;;) {
            VTRY("vhm poisson", cudaMemsetAsync(nact, 0, sizeof(int), st));
            for (int k = 0; k < CHUNK; ++k) {
                k_cg_apply<<<nbv, VT, 0, st>>>(op, K, B.p, B.q, B.partial);
                k_col_sum<<<K, VT, 0, st>>>(K, nbv, B.partial, pq);
                k_cg_alpha<<<vblk(K), VT, 0, st>>>(K, rz, pq, active, alpha);
                k_cg_step<<<nbv, VT, 0, st>>>(op, K, alpha, B.p, B.q, B.x, B.r, B.z, B.partial);
                k_col_sum<<<K, VT, 0, st>>>(K, nbv, B.partial, rzn);
                if (k == CHUNK - 1) VTRY("vhm poisson", cudaMemsetAsync(nact, 0, sizeof(int), st));
                k_cg_beta<<<vblk(K), VT, 0, st>>>(K, 1e-28, rz0, rz, rzn, active, beta, nact);
                k_cg_dir<<<nbv, VT, 0, st>>>(op, K, active, beta, B.z, B.p);
            }
            VTRY("vhm poisson", cudaGetLastError());
            cg += CHUNK;
            int ha = 0;
            VTRY("vhm poisson", cudaMemcpyAsync(&ha, nact, sizeof(int), cudaMemcpyDeviceToHost, st));
            VTRY("vhm poisson", cudaStreamSynchronize(st));
            if (!ha) break;
            if (cg >= MAX_CG) { c->err = "vhm: Poisson solve did not converge"; return CSS_ERR_ITER_LIMIT; }
        }
        iters_cg += cg;
        // ---- targets: distance, tangent, kept pairs in j order
        k_evaluate<<<vblk((int64_t)ns * n), VT, 0, st>>>(op, K, ns, n, B.src, parts->face, parts->bary, B.x, Y, r_c,
                                                         B.od, B.ot, B.keep);
        k_count_rows<<<ns, VT, 0, st>>>(n, B.keep, B.cnt);
        VTRY("vhm evaluate", cudaGetLastError());
        std::vector<int64_t> hc(ns);
        VTRY("vhm evaluate", cudaMemcpyAsync(hc.data(), B.cnt, ns * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        VTRY("vhm evaluate", cudaStreamSynchronize(st));
        int64_t bt = 0;
        std::vector<int64_t> off(ns);
        for (int s = 0; s < ns; ++s) {
            off[s] = total + bt;
            rows[s0 + s] = total + bt;
            bt += hc[s];
        }
        if (total + bt <= capacity && bt > 0 && nbr_j && dist && tangent) {
            int32_t* oj = nbr_j;
            double *odd = dist, *ott = tangent;
            Batch S;
            if (!dev_out) {   // stage this batch's rows, then copy them to the host arrays
                VTRY("vhm output", S.get(&oj, (size_t)bt));
                VTRY("vhm output", S.get(&odd, (size_t)bt));
                VTRY("vhm output", S.get(&ott, 3 * (size_t)bt));
                for (int s = 0; s < ns; ++s) off[s] -= total;
            }
            VTRY("vhm output", cudaMemcpyAsync(B.roff, off.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, st));
            k_compact_rows<<<ns, VT, 0, st>>>(n, B.keep, B.od, B.ot, B.roff, oj, odd, ott);
            VTRY("vhm output", cudaGetLastError());
            if (!dev_out) {
                VTRY("vhm output", cudaMemcpyAsync(nbr_j + total, oj, bt * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                VTRY("vhm output", cudaMemcpyAsync(dist + total, odd, bt * sizeof(double), cudaMemcpyDeviceToHost, st));
                VTRY("vhm output", cudaMemcpyAsync(tangent + 3 * total, ott, 3 * bt * sizeof(double),
                                                   cudaMemcpyDeviceToHost, st));
            }
            VTRY("vhm output", cudaStreamSynchronize(st));
        }
        total += bt;
    }
    rows[n] = total;
    *n_pairs = total;
    c->last_counters[0] = n;
    c->last_counters[1] = iters_heat;
    c->last_counters[2] = iters_cg;
    c->last_counters[3] = total;
    c->last_counters[4] = (n + K - 1) / K;
    c->last_counters[5] = K;
    if (total > capacity) { c->err = "vhm_neighbors: capacity too small"; return CSS_ERR_CAPACITY; }
    if (!row_start || (total > 0 && (!nbr_j || !dist || !tangent))) return CSS_ERR_INVALID_ARG;
    if (dev_ptr(row_start)) {
        VTRY("vhm output", cudaMemcpyAsync(row_start, rows.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        VTRY("vhm output", cudaStreamSynchronize(st));
    } else {
        std::copy(rows.begin(), rows.end(), row_start);
    }
    return CSS_OK;
}
