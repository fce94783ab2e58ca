// mesh_prep.cu -- device-side intrinsic preparation of an uploaded mesh (Sec. 2.2).
//
// Topology: every half-edge inserts its (min, max) vertex key into an open
// addressing table; two inserters of one key are twins, one is a boundary edge,
// three or more make the mesh non-manifold.  Geometry: per-face planar layout
// (minimum-image edge vectors on periodic meshes), per-half-edge frame and the
// rotations into the two neighbouring frames, vertex angle sums (summed over the
// sorted one-ring, so the result does not depend on thread timing).  Faces are also
// ranked along a Morton curve through their first corners: particle buckets are kept in
// that order, so sources processed at the same time sit close together and their
// patches share the L2.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "css_internal.h"

namespace {

using css::HeRec;

constexpr unsigned long long EMPTY = ~0ull;
constexpr double TWO_PI = 6.283185307179586476925286766559;

struct TopoTab {
    unsigned long long* key;
    int32_t* cnt;
    int32_t* h0;
    int32_t* h1;
    int logcap;
};

__global__ void k_check_faces(const int32_t* F, int64_t nf, int64_t nv, int* flag) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int32_t a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) atomicOr(flag, 1);
    else if (a == b || b == c || a == c) atomicOr(flag, 2);
}

__global__ void k_check_verts(const double* X, int64_t nv, int* flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * nv) return;
    if (!isfinite(X[i])) atomicOr(flag, 1);
}

__global__ void k_topo_insert(const int32_t* F, int64_t nf, TopoTab t, int* flag) {
    int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (h >= 3 * nf) return;
    int64_t f = h / 3;
    int k = (int)(h % 3);
    uint32_t a = (uint32_t)F[h], b = (uint32_t)F[3 * f + (k + 1) % 3];
    uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
    unsigned long long want = ((unsigned long long)lo << 32) | hi;
    uint64_t mix = want * 0x9E3779B97F4A7C15ull;
    uint32_t mask = (1u << t.logcap) - 1u;
    uint32_t slot = (uint32_t)(mix >> (64 - t.logcap));
    for (uint32_t p = 0; p <= mask; ++p) {
        unsigned long long prev = atomicCAS(t.key + slot, EMPTY, want);
        if (prev == EMPTY || prev == want) {
            int c = atomicAdd(t.cnt + slot, 1);
            if (c == 0) t.h0[slot] = (int32_t)h;
            else if (c == 1) t.h1[slot] = (int32_t)h;
            else atomicOr(flag, 4);
            return;
        }
        slot = (slot + 1u) & mask;
    }
    atomicOr(flag, 8);
}

__global__ void k_topo_link(const int32_t* F, TopoTab t, int32_t* twin, int32_t* edge, int* flag,
                            unsigned long long* n_edges) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= (1ll << t.logcap)) return;
    int c = t.cnt[s];
    if (c == 0) return;
    atomicAdd(n_edges, 1ull);
    int32_t h0 = t.h0[s];
    if (c == 1) { twin[h0] = -1; edge[h0] = h0; return; }
    if (c > 2) return;
    int32_t h1 = t.h1[s];
    if (F[h0] == F[h1]) atomicOr(flag, 16);   // both run a->b: inconsistent orientation
    twin[h0] = h1; twin[h1] = h0;
    int32_t e = h0 < h1 ? h0 : h1;
    edge[h0] = e; edge[h1] = e;
}

__device__ void min_image(double* d, int periodic, double px, double py) {
    if (!periodic) return;
    d[0] -= px * floor(d[0] / px + 0.5);
    d[1] -= py * floor(d[1] / py + 0.5);
}

__global__ void k_faces(const double* X, const int32_t* F, int64_t nf, int periodic, double px, double py,
                        double* lay, double* frame, int* flag) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const double* x0 = X + 3 * (int64_t)F[3 * f];
    const double* x1 = X + 3 * (int64_t)F[3 * f + 1];
    const double* x2 = X + 3 * (int64_t)F[3 * f + 2];
    double a[3], b[3];
    for (int c = 0; c < 3; ++c) { a[c] = x1[c] - x0[c]; b[c] = x2[c] - x0[c]; }
    min_image(a, periodic, px, py);
    min_image(b, periodic, px, py);
    double La = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(nn > 0.0) || !(La > 0.0)) { atomicOr(flag, 32); return; }
    double e1[3] = {a[0] / La, a[1] / La, a[2] / La};
    for (int c = 0; c < 3; ++c) n[c] /= nn;
    double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
    lay[3 * f] = La;
    lay[3 * f + 1] = b[0] * e1[0] + b[1] * e1[1] + b[2] * e1[2];
    lay[3 * f + 2] = b[0] * e2[0] + b[1] * e2[1] + b[2] * e2[2];
    for (int c = 0; c < 3; ++c) {
        frame[9 * f + c] = x0[c];
        frame[9 * f + 3 + c] = e1[c];
        frame[9 * f + 6 + c] = e2[c];
    }
}

__global__ void k_halfedges(const double* lay, const int32_t* F, const int32_t* twin, int64_t nf, HeRec* he,
                            css::HeRec32* he32, float* lay32, uint8_t* bnd, int32_t* ring_cnt) {
    int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (h >= 3 * nf) return;
    int64_t f = h / 3;
    int k = (int)(h % 3);
    double P[3][2] = {{0.0, 0.0}, {lay[3 * f], 0.0}, {lay[3 * f + 1], lay[3 * f + 2]}};
    const double* A = P[k];
    const double* B = P[(k + 1) % 3];
    const double* C = P[(k + 2) % 3];
    double ex = B[0] - A[0], ey = B[1] - A[1];
    double L = sqrt(ex * ex + ey * ey);
    double dx = ex / L, dy = ey / L;
    double wx = C[0] - A[0], wy = C[1] - A[1];
    HeRec r;
    r.L = L;
    r.cx = wx * dx + wy * dy;
    r.cy = dx * wy - dy * wx;
    double Lc = sqrt(r.cx * r.cx + r.cy * r.cy);
    r.cl = r.cx / Lc;
    r.sl = r.cy / Lc;
    double qx = L - r.cx, qy = -r.cy;
    double Ld = sqrt(qx * qx + qy * qy);
    r.cr = qx / Ld;
    r.sr = qy / Ld;
    r.tl = twin[3 * f + (k + 2) % 3];
    r.tr = twin[3 * f + (k + 1) % 3];
    he[h] = r;
    css::HeRec32 q;
    q.L = (float)r.L; q.cx = (float)r.cx; q.cy = (float)r.cy;
    q.cl = (float)r.cl; q.sl = (float)r.sl; q.cr = (float)r.cr; q.sr = (float)r.sr;
    q.pad = 0;
    he32[h] = q;
    lay32[h] = (float)lay[h];   // 3 per face: the same indexing as the half-edges
    if (twin[h] < 0) { bnd[F[h]] = 1; bnd[F[3 * f + (k + 1) % 3]] = 1; }
    atomicAdd(ring_cnt + F[h], 1);
}

__global__ void k_ring_scatter(const int32_t* F, int64_t nf, const int32_t* ring_start, int32_t* fill, int32_t* ring) {
    int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (h >= 3 * nf) return;
    int32_t v = F[h];
    int p = atomicAdd(fill + v, 1);
    ring[ring_start[v] + p] = (int32_t)h;
}

// sort each ring by half-edge id (deterministic order), sum corner angles, set flags
// Angle sum of every vertex and its pseudo-source flag (boundary, flat or saddle); and the
// cumulative angle of every corner around its vertex: starting from the corner of smallest
// half-edge id, corners follow counter-clockwise (the next corner is the one across the edge
// the current corner ends on), each at the sum of the widths before it.  A ring that is not
// one closed fan (boundary, non-manifold vertex) gets NaN.
__global__ void k_vertices(int64_t nv, const int32_t* ring_start, int32_t* ring, const HeRec* he,
                           const int32_t* twin, double* theta, const uint8_t* bnd, uint8_t* pseudo, float2* cang,
                           unsigned long long* n_pseudo) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int s = ring_start[v], e = ring_start[v + 1];
    for (int i = s + 1; i < e; ++i) {
        int32_t x = ring[i];
        int j = i - 1;
        while (j >= s && ring[j] > x) { ring[j + 1] = ring[j]; --j; }
        ring[j + 1] = x;
    }
    double th = 0.0;
    for (int i = s; i < e; ++i) {
        const HeRec& r = he[ring[i]];
        th += atan2(r.cy, r.cx);   // corner angle at the origin corner of this half-edge
    }
    theta[v] = th;
    uint8_t p = (uint8_t)(bnd[v] || th >= TWO_PI - 1e-9);
    pseudo[v] = p;
    if (p) atomicAdd(n_pseudo, 1ull);
    bool closed = false;
    if (!bnd[v] && e > s) {
        const int32_t h0 = ring[s];
        int32_t h = h0;
        double cum = 0.0;
        int steps = 0;
        while (steps < e - s) {
            const HeRec& r = he[h];
            const double w = atan2(r.cy, r.cx);
            cang[h] = make_float2((float)cum, (float)w);
            cum += w;
            ++steps;
            const int32_t f = h / 3, k = h - 3 * f;
            const int32_t nh = twin[3 * f + (k == 0 ? 2 : k - 1)];   // the corner across the edge c -> v
            if (nh < 0) break;
            h = nh;
            if (h == h0) { closed = true; break; }
        }
        closed = closed && steps == e - s;
    }
    if (!closed)
        for (int i = s; i < e; ++i) cang[ring[i]] = make_float2(NAN, NAN);
}

inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

namespace {
// first corner of every face (world), for the face ranking
__global__ void k_origin(const double* frame, int64_t nf, float* out) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    out[3 * f] = (float)frame[9 * f];
    out[3 * f + 1] = (float)frame[9 * f + 1];
    out[3 * f + 2] = (float)frame[9 * f + 2];
}

uint32_t spread10(uint32_t v) {   // 10 bits to every third of 30
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
}  // namespace

css::DMesh css_mesh::view() const {
    css::DMesh d;
    d.nv = (int32_t)nv;
    d.nf = (int32_t)nf;
    d.periodic = periodic;
    d.per[0] = per[0];
    d.per[1] = per[1];
    d.he = he;
    d.twin = twin;
    d.edge = edge;
    d.fv = fv;
    d.lay = lay;
    d.frame = frame;
    d.theta = theta;
    d.pseudo = pseudo;
    d.bnd = bnd;
    d.ring_start = ring_start;
    d.ring = ring;
    d.he32 = he32;
    d.lay32 = lay32;
    d.frank = frank;
    d.cang = cang;
    return d;
}

namespace cssi {

#define CK(x)                                                    \
    do {                                                         \
        cudaError_t e_ = (x);                                    \
        if (e_ != cudaSuccess) {                                 \
            ctx->err = std::string("mesh_upload: ") + cudaGetErrorString(e_); \
            rc = (e_ == cudaErrorMemoryAllocation) ? CSS_ERR_OOM : CSS_ERR_CUDA; \
            goto done;                                           \
        }                                                        \
    } while (0)

int build_mesh(css_ctx* ctx, const double* dX, int64_t nv, const int32_t* dF, int64_t nf, const double* period,
               css_mesh* m) {
    int rc = CSS_OK;
    cudaStream_t st = ctx->stream;
    const int64_t nh = 3 * nf;
    int logcap = 4;
    while ((1ll << logcap) < 2 * nh) ++logcap;
    const int64_t cap = 1ll << logcap;
    TopoTab t{};
    t.logcap = logcap;
    int* dflag = nullptr;
    unsigned long long* dcnt = nullptr;
    int32_t* ring_cnt = nullptr;
    int32_t* tmp = nullptr;
    int hflag = 0;
    unsigned long long hcnt[2] = {0, 0};
    m->nv = nv;
    m->nf = nf;
    if (period) { m->periodic = 1; m->per[0] = period[0]; m->per[1] = period[1]; }
    CK(cudaMalloc(&t.key, cap * sizeof(unsigned long long)));
    CK(cudaMalloc(&t.cnt, cap * sizeof(int32_t)));
    CK(cudaMalloc(&t.h0, cap * sizeof(int32_t)));
    CK(cudaMalloc(&t.h1, cap * sizeof(int32_t)));
    CK(cudaMalloc(&dflag, sizeof(int)));
    CK(cudaMalloc(&dcnt, 2 * sizeof(unsigned long long)));
    CK(cudaMalloc(&m->he, nh * sizeof(HeRec)));
    CK(cudaMalloc(&m->twin, nh * sizeof(int32_t)));
    CK(cudaMalloc(&m->edge, nh * sizeof(int32_t)));
    CK(cudaMalloc(&m->fv, nh * sizeof(int32_t)));
    CK(cudaMalloc(&m->lay, 3 * nf * sizeof(double)));
    CK(cudaMalloc(&m->frame, 9 * nf * sizeof(double)));
    CK(cudaMalloc(&m->theta, nv * sizeof(double)));
    CK(cudaMalloc(&m->pseudo, nv));
    CK(cudaMalloc(&m->bnd, nv));
    CK(cudaMalloc(&m->ring_start, (nv + 1) * sizeof(int32_t)));
    CK(cudaMalloc(&m->ring, nh * sizeof(int32_t)));
    CK(cudaMalloc(&m->X, 3 * nv * sizeof(double)));
    CK(cudaMalloc(&m->he32, nh * sizeof(css::HeRec32)));
    CK(cudaMalloc(&m->lay32, 3 * nf * sizeof(float)));
    CK(cudaMalloc(&m->frank, nf * sizeof(int32_t)));
    CK(cudaMalloc(&m->cang, nh * sizeof(float2)));
    CK(cudaMalloc(&ring_cnt, (nv + 1) * sizeof(int32_t)));
    CK(cudaMalloc(&tmp, scan_tmp_ints(nv + 1) * sizeof(int32_t)));
    CK(cudaMemcpyAsync(m->X, dX, 3 * nv * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(m->fv, dF, nh * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(t.key, 0xff, cap * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(t.cnt, 0, cap * sizeof(int32_t), st));
    CK(cudaMemsetAsync(dflag, 0, sizeof(int), st));
    CK(cudaMemsetAsync(dcnt, 0, 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(m->bnd, 0, nv, st));
    CK(cudaMemsetAsync(ring_cnt, 0, (nv + 1) * sizeof(int32_t), st));
    k_check_faces<<<nblk(nf), 256, 0, st>>>(dF, nf, nv, dflag);
    k_check_verts<<<nblk(3 * nv), 256, 0, st>>>(dX, nv, dflag);
    CK(cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hflag & 1) { ctx->err = "mesh_upload: vertex index out of range or non-finite coordinate"; rc = CSS_ERR_INVALID_ARG; goto done; }
    if (hflag & 2) { ctx->err = "mesh_upload: face with a repeated vertex"; rc = CSS_ERR_NONMANIFOLD; goto done; }
    k_topo_insert<<<nblk(nh), 256, 0, st>>>(dF, nf, t, dflag);
    k_topo_link<<<nblk(cap), 256, 0, st>>>(dF, t, m->twin, m->edge, dflag, dcnt);
    k_faces<<<nblk(nf), 256, 0, st>>>(dX, dF, nf, m->periodic, m->per[0], m->per[1], m->lay, m->frame, dflag);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hflag & (4 | 8)) { ctx->err = "mesh_upload: an edge is shared by more than two faces"; rc = CSS_ERR_NONMANIFOLD; goto done; }
    if (hflag & 16) { ctx->err = "mesh_upload: inconsistent face orientation"; rc = CSS_ERR_NONMANIFOLD; goto done; }
    if (hflag & 32) { ctx->err = "mesh_upload: degenerate (zero-area) face"; rc = CSS_ERR_NONMANIFOLD; goto done; }
    k_halfedges<<<nblk(nh), 256, 0, st>>>(m->lay, dF, m->twin, nf, m->he, m->he32, m->lay32, m->bnd, ring_cnt);
    CK(launch_scan_i32(ring_cnt, m->ring_start, nv + 1, tmp, st));
    CK(cudaMemsetAsync(ring_cnt, 0, (nv + 1) * sizeof(int32_t), st));
    k_ring_scatter<<<nblk(nh), 256, 0, st>>>(dF, nf, m->ring_start, ring_cnt, m->ring);
    k_vertices<<<nblk(nv), 256, 0, st>>>(nv, m->ring_start, m->ring, m->he, m->twin, m->theta, m->bnd, m->pseudo,
                                         m->cang, dcnt + 1);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(hcnt, dcnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    m->ne = (int64_t)hcnt[0];
    m->npseudo = (int64_t)hcnt[1];
    {   // Morton rank of every face (host sort, once per mesh)
        float* dorg = nullptr;
        CK(cudaMalloc(&dorg, 3 * nf * sizeof(float)));
        k_origin<<<nblk(nf), 256, 0, st>>>(m->frame, nf, dorg);
        std::vector<float> org(3 * nf);
        cudaError_t e = cudaMemcpyAsync(org.data(), dorg, 3 * nf * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(dorg);
        CK(e);
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t f = 0; f < nf; ++f)
            for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], org[3 * f + a]); hi[a] = std::max(hi[a], org[3 * f + a]); }
        std::vector<uint64_t> key(nf);
        for (int64_t f = 0; f < nf; ++f) {
            uint32_t code = 0;
            for (int a = 0; a < 3; ++a) {
                const float ext = hi[a] - lo[a];
                const uint32_t q = ext > 0.f ? (uint32_t)std::min(1023.f, (org[3 * f + a] - lo[a]) / ext * 1024.f) : 0u;
                code |= spread10(q) << a;
            }
            key[f] = ((uint64_t)code << 32) | (uint64_t)f;
        }
        std::sort(key.begin(), key.end());
        std::vector<int32_t> rank(nf);
        for (int64_t r = 0; r < nf; ++r) rank[(int64_t)(key[r] & 0xffffffffu)] = (int32_t)r;
        CK(cudaMemcpyAsync(m->frank, rank.data(), nf * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
done:
    cudaFree(t.key);
    cudaFree(t.cnt);
    cudaFree(t.h0);
    cudaFree(t.h1);
    cudaFree(dflag);
    cudaFree(dcnt);
    cudaFree(ring_cnt);
    cudaFree(tmp);
    return rc;
}

}  // namespace cssi
