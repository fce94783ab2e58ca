// api.cu -- the C ABI declared in include/css.h.
//
// Host-side runtime: argument checking, staging of host/device pointers, the
// neighbour/force workspace (sized from the occupancy of the persistent kernel and
// grown when a launch reports an overflow), CSR output, CUDA-graph capture of the
// per-step kernel sequence, and the batched multi-mesh driver.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "css_internal.h"

using cssi::GeoJob;
using cssi::GeoWs;

namespace {

constexpr int MAX_RETRY = 8;
constexpr int WIN_CAP_MAX = 1 << 20;

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int cuda_fail(css_ctx* c, const char* what, cudaError_t e) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CSS_ERR_OOM : CSS_ERR_CUDA;
}

#define TRY(ctx, what, x)                                  \
    do {                                                   \
        cudaError_t e__ = (x);                             \
        if (e__ != cudaSuccess) return cuda_fail(ctx, what, e__); \
    } while (0)

// copy n elements from a host or device pointer into a fresh device buffer
template <class T>
cudaError_t stage_in(const T* src, size_t n, T** dst, cudaStream_t st) {
    *dst = nullptr;
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(*dst, src, n * sizeof(T), is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
}

template <class T>
cudaError_t copy_out(T* dst, const T* dsrc, size_t n, cudaStream_t st) {
    if (!dst || n == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, dsrc, n * sizeof(T), is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
}

int next_pow2(int x) {
    int p = 64;
    while (p < x) p <<= 1;
    return p;
}

// ---- workspace for the persistent neighbour/force kernel
int ensure_ws(css_ctx* c, int precision, int shared, GeoWs* out, int* nctas) {
    int bps = cssi::geodesic_blocks_per_sm(precision, c->warps_per_cta, shared);
    if (bps < 1) bps = 1;
    const int ncta = c->sm_count * bps;
    const int nwarps = ncta * c->warps_per_cta;
    GeoWs g{};
    g.shared = shared;
    g.stride = cssi::geo_ws_bytes_per_warp(precision, c->win_cap, &g.log_eh, &g.log_vh, &g.log_fh, &g.fcap, &g.emcap);
    g.wcap = c->win_cap;
    g.nwarps = nwarps;
    const size_t need = g.stride * (size_t)nwarps;
    // a layout change re-zeroes the workspace so old bytes never look like valid hash tags
    const int64_t key = (int64_t)precision * 1000003 + (int64_t)c->win_cap * 31 + c->warps_per_cta + 17 * shared;
    const bool relayout = (need > c->ws_bytes) || (c->ws_warps < nwarps) || (c->ws_key != key);
    if (need > c->ws_bytes) {
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
        TRY(c, "workspace", cudaMalloc(&c->ws, need));
        c->ws_bytes = need;
    }
    if (c->ws_warps < nwarps) {
        cudaFree(c->ws_gen);
        c->ws_gen = nullptr;
        TRY(c, "workspace", cudaMalloc(&c->ws_gen, nwarps * sizeof(uint32_t)));
        c->ws_warps = nwarps;
    }
    if (relayout) {
        TRY(c, "workspace", cudaMemsetAsync(c->ws, 0, c->ws_bytes, c->stream));
        TRY(c, "workspace", cudaMemsetAsync(c->ws_gen, 0, c->ws_warps * sizeof(uint32_t), c->stream));
        c->ws_key = key;
    }
    g.base = (char*)c->ws;
    g.gen = c->ws_gen;
    *out = g;
    *nctas = ncta;
    return CSS_OK;
}

int ensure_pairs(css_parts* p, int cap) {
    css_ctx* c = p->ctx;
    if (p->pair_cap_alloc >= cap && p->pj) return CSS_OK;
    cudaFree(p->pj); cudaFree(p->pd); cudaFree(p->pt);
    p->pj = nullptr; p->pd = nullptr; p->pt = nullptr; p->pair_cap_alloc = 0;
    const size_t n = (size_t)p->n * cap;
    TRY(c, "pair slab", cudaMalloc(&p->pj, std::max<size_t>(n, 1) * sizeof(int32_t)));
    TRY(c, "pair slab", cudaMalloc(&p->pd, std::max<size_t>(n, 1) * sizeof(double)));
    TRY(c, "pair slab", cudaMalloc(&p->pt, std::max<size_t>(3 * n, 1) * sizeof(double)));
    p->pair_cap_alloc = cap;
    return CSS_OK;
}

GeoJob make_job(css_parts* p, double rc, int want_pairs, int want_forces, const css_potential* pot) {
    GeoJob j{};
    j.m = p->mesh->view();
    j.n = (int32_t)p->n;
    j.face = p->face;
    j.bary = p->bary;
    j.fstart = p->fstart;
    j.fitems = p->fitems;
    j.order = nullptr;
    j.rc = rc;
    j.want_pairs = want_pairs;
    j.pair_cap = p->pair_cap_alloc;
    j.pcnt = p->pcnt;
    j.pj = p->pj;
    j.pd = p->pd;
    j.pt = p->pt;
    j.want_forces = want_forces;
    if (pot) j.pot = *pot;
    j.force = p->force;
    j.epot = p->ctx->depot;
    return j;
}

// record a timing event on the context stream (also inside a graph capture)
cudaError_t record_ev(css_ctx* c, cudaEvent_t ev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->stream, &cs);
    c->ev_valid = 1;
    if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ev, c->stream, cudaEventRecordExternal);
    return cudaEventRecord(ev, c->stream);
}

// one bucket + neighbour/force launch (no synchronisation)
int enqueue_geo(css_parts* p, double rc, int prec, int want_pairs, int want_forces, const css_potential* pot,
                const GeoWs& g, int nctas) {
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    TRY(c, "bucket", cssi::launch_bucket((int32_t)p->n, (int32_t)p->mesh->nf, p->face, p->fcnt, p->fstart, p->fitems,
                                         p->scan_tmp, st));
    TRY(c, "reset", cudaMemsetAsync(c->dscal, 0, sizeof(int), st));
    GeoJob j = make_job(p, rc, want_pairs, want_forces, pot);
    TRY(c, "event", record_ev(c, c->ev_geo0));
    TRY(c, "geodesic", cssi::launch_geodesic(j, nullptr, nullptr, nullptr, (int32_t)p->n, prec, g, c->warps_per_cta,
                                             nctas, c->dscal, c->dscal + 1, c->dcount, st));
    TRY(c, "event", record_ev(c, c->ev_geo1));
    return CSS_OK;
}

int read_status(css_ctx* c, int* status) {
    TRY(c, "status", cudaMemcpyAsync(c->hstat, c->dscal + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    TRY(c, "status", cudaMemcpyAsync(c->hcount, c->dcount, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    TRY(c, "sync", cudaStreamSynchronize(c->stream));
    *status = *c->hstat;
    for (int k = 0; k < 4; ++k) c->last_counters[k] = (int64_t)c->hcount[k];
    return CSS_OK;
}

// grow the capacity that overflowed; false when nothing can grow any more.  A table
// overflow of a launch with shared-memory tables sets *to_global instead: the patch is
// too large for them and the launch is repeated with the global tables.
bool grow_for(css_ctx* c, int status, int* retries, int shared, bool* to_global) {
    ++*retries;
    *to_global = false;
    if (*retries > MAX_RETRY) return false;
    bool grown = false;
    if ((status & css::ST_HASH_OVERFLOW) && shared) { *to_global = true; grown = true; status &= ~css::ST_HASH_OVERFLOW; }
    if (status & (css::ST_WIN_OVERFLOW | css::ST_HASH_OVERFLOW | css::ST_ITER_LIMIT)) {
        if (c->win_cap >= WIN_CAP_MAX) return false;
        c->win_cap *= 2;
        grown = true;
    }
    if (status & css::ST_PAIR_OVERFLOW) { c->pair_cap *= 2; grown = true; }
    return grown;
}

int use_shared(const css_parts* p) { return p->ctx->shared_tables && !p->global_tables; }

int status_error(css_ctx* c, int status) {
    if (status & (css::ST_WIN_OVERFLOW | css::ST_HASH_OVERFLOW)) {
        c->err = "window workspace exhausted (capacity " + std::to_string(c->win_cap) + ")";
        return CSS_ERR_QUEUE_OVERFLOW;
    }
    if (status & (css::ST_ITER_LIMIT | css::ST_WALK_LIMIT)) { c->err = "device loop reached its iteration cap"; return CSS_ERR_ITER_LIMIT; }
    if (status & css::ST_PIECES) { c->err = "window trimming produced too many pieces"; return CSS_ERR_QUEUE_OVERFLOW; }
    if (status & css::ST_PAIR_OVERFLOW) { c->err = "pair slab overflow"; return CSS_ERR_QUEUE_OVERFLOW; }
    c->err = "device status " + std::to_string(status);
    return CSS_ERR_CUDA;
}

// synchronous neighbour / force evaluation with overflow retries
int run_geo(css_parts* p, double rc, int prec, int want_pairs, int want_forces, const css_potential* pot) {
    css_ctx* c = p->ctx;
    int retries = 0;
    TRY(c, "reset", cudaMemsetAsync(c->dcount, 0, 8 * sizeof(unsigned long long), c->stream));
    for (;;) {
        if (want_pairs) { int rc2 = ensure_pairs(p, c->pair_cap); if (rc2) return rc2; }
        GeoWs g;
        int nctas = 0;
        const int shared = use_shared(p);
        int rc1 = ensure_ws(c, prec, shared, &g, &nctas);
        if (rc1) return rc1;
        TRY(c, "reset", cudaMemsetAsync(c->dscal + 1, 0, sizeof(int), c->stream));
        TRY(c, "reset", cudaMemsetAsync(c->depot, 0, sizeof(double), c->stream));
        rc1 = enqueue_geo(p, rc, prec, want_pairs, want_forces, pot, g, nctas);
        if (rc1) return rc1;
        int status = 0;
        rc1 = read_status(c, &status);
        if (rc1) return rc1;
        if (status == 0) return CSS_OK;
        c->last_counters[4] += 1;
        bool to_global = false;
        if (!grow_for(c, status, &retries, shared, &to_global)) return status_error(c, status);
        if (to_global) p->global_tables = 1;
    }
}

bool finite_all(const double* h, size_t n) {
    for (size_t i = 0; i < n; ++i) if (!std::isfinite(h[i])) return false;
    return true;
}

}  // namespace

// =====================================================================================
// C ABI (declared extern "C" in css.h, so these definitions have C linkage)
static bool bad_prec(int prec) { return prec != CSS_FP64 && prec != CSS_FP32; }
static bool bad_rc(double rc) { return !(rc > 0.0); }   // INFINITY allowed, NaN rejected

int css_create(css_ctx** out, int device, void* stream) {
    if (!out) return CSS_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) { cudaGetLastError(); return CSS_ERR_NO_DEVICE; }
    if (device < 0 || device >= ndev) return CSS_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return CSS_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return CSS_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return CSS_ERR_NO_DEVICE;   // built for sm_103a only
    css_ctx* c = new css_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (!c->stream) {   // graph capture needs a real stream: own one
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return CSS_ERR_CUDA; }
        c->own_stream = 1;
    }
    c->sm_count = prop.multiProcessorCount;
    if (cudaMalloc(&c->dscal, 4 * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->dcount, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->depot, sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->hstat, 4 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->hcount, 8 * sizeof(unsigned long long)) != cudaSuccess) {
        css_destroy(c);
        return CSS_ERR_OOM;
    }
    if (cudaEventCreate(&c->ev_geo0) != cudaSuccess || cudaEventCreate(&c->ev_geo1) != cudaSuccess) {
        css_destroy(c);
        return CSS_ERR_CUDA;
    }
    cudaMemset(c->dscal, 0, 4 * sizeof(int));
    cudaMemset(c->dcount, 0, 8 * sizeof(unsigned long long));
    *out = c;
    return CSS_OK;
}

int css_destroy(css_ctx* c) {
    if (!c) return CSS_ERR_INVALID_ARG;
    cudaFree(c->ws);
    cudaFree(c->ws_gen);
    cudaFree(c->dscal);
    cudaFree(c->dcount);
    cudaFree(c->depot);
    cudaFreeHost(c->hstat);
    cudaFreeHost(c->hcount);
    if (c->ev_geo0) cudaEventDestroy(c->ev_geo0);
    if (c->ev_geo1) cudaEventDestroy(c->ev_geo1);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return CSS_OK;
}

const char* css_last_error(const css_ctx* c) { return c ? c->err.c_str() : "null context"; }

int css_last_counters(const css_ctx* c, int64_t out[6]) {
    if (!c || !out) return CSS_ERR_INVALID_ARG;
    out[0] = c->last_counters[0];
    out[1] = c->last_counters[1];
    out[2] = c->last_counters[2];
    out[3] = c->last_counters[3];
    out[4] = 0;
    out[5] = c->last_counters[4];
    return CSS_OK;
}

int css_last_kernel_ms(css_ctx* c, double* ms) {
    if (!c || !ms || !c->ev_valid) return CSS_ERR_INVALID_ARG;
    float f = 0.f;
    TRY(c, "kernel timing", cudaEventSynchronize(c->ev_geo1));
    TRY(c, "kernel timing", cudaEventElapsedTime(&f, c->ev_geo0, c->ev_geo1));
    *ms = (double)f;
    return CSS_OK;
}

int css_fma_peak(css_ctx* c, int precision, double* flops_per_s) {
    if (!c || !flops_per_s || bad_prec(precision)) return CSS_ERR_INVALID_ARG;
    TRY(c, "fma peak", cssi::measure_fma_peak(precision, c->sm_count, c->stream, flops_per_s));
    return CSS_OK;
}

int css_set_launch(css_ctx* c, int32_t warps_per_cta, int32_t window_capacity) {
    if (!c || warps_per_cta < 0 || warps_per_cta > 8 || window_capacity < 0) return CSS_ERR_INVALID_ARG;
    if (warps_per_cta) c->warps_per_cta = warps_per_cta;
    if (window_capacity) c->win_cap = next_pow2(window_capacity);
    return CSS_OK;
}

int css_mesh_upload(css_ctx* c, const double* verts, int64_t nv, const int32_t* faces, int64_t nf, const double* period,
                    css_mesh** out) {
    if (!c || !out || !verts || !faces || nv < 3 || nf < 1 || nv > INT32_MAX / 2 || nf > INT32_MAX / 6)
        return CSS_ERR_INVALID_ARG;
    if (period && !(period[0] > 0.0 && period[1] > 0.0)) return CSS_ERR_INVALID_ARG;
    *out = nullptr;
    double* dX = nullptr;
    int32_t* dF = nullptr;
    cudaError_t e = stage_in(verts, 3 * (size_t)nv, &dX, c->stream);
    if (e == cudaSuccess) e = stage_in(faces, 3 * (size_t)nf, &dF, c->stream);
    if (e != cudaSuccess) { cudaFree(dX); cudaFree(dF); return cuda_fail(c, "mesh_upload", e); }
    css_mesh* m = new css_mesh();
    m->ctx = c;
    int rc = cssi::build_mesh(c, dX, nv, dF, nf, period, m);
    cudaFree(dX);
    cudaFree(dF);
    if (rc) { css_mesh_free(m); return rc; }
    *out = m;
    return CSS_OK;
}

int css_mesh_free(css_mesh* m) {
    if (!m) return CSS_ERR_INVALID_ARG;
    cudaFree(m->he); cudaFree(m->twin); cudaFree(m->edge); cudaFree(m->fv); cudaFree(m->lay);
    cudaFree(m->frame); cudaFree(m->theta); cudaFree(m->pseudo); cudaFree(m->bnd);
    cudaFree(m->ring_start); cudaFree(m->ring); cudaFree(m->X); cudaFree(m->he32); cudaFree(m->lay32);
    delete m;
    return CSS_OK;
}

int css_mesh_counts(const css_mesh* m, int64_t out[4]) {
    if (!m || !out) return CSS_ERR_INVALID_ARG;
    out[0] = m->nv; out[1] = m->nf; out[2] = m->ne; out[3] = m->npseudo;
    return CSS_OK;
}

int css_particles_set(css_ctx* c, css_mesh* m, int64_t n, const int32_t* face, const double* bary, const double* vel,
                      const double* orient, uint64_t seed, css_parts** out) {
    if (!c || !m || !out || !face || !bary || n < 1 || n > INT32_MAX / 64) return CSS_ERR_INVALID_ARG;
    *out = nullptr;
    // validation on the host (a copy when the input is on the device)
    std::vector<int32_t> hf(n);
    std::vector<double> hb(3 * n);
    if (is_device_ptr(face)) cudaMemcpy(hf.data(), face, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
    else memcpy(hf.data(), face, n * sizeof(int32_t));
    if (is_device_ptr(bary)) cudaMemcpy(hb.data(), bary, 3 * n * sizeof(double), cudaMemcpyDeviceToHost);
    else memcpy(hb.data(), bary, 3 * n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        if (hf[i] < 0 || hf[i] >= m->nf) { c->err = "particles_set: face index out of range"; return CSS_ERR_INVALID_ARG; }
        const double s = hb[3 * i] + hb[3 * i + 1] + hb[3 * i + 2];
        if (!finite_all(&hb[3 * i], 3) || fabs(s - 1.0) > 1e-9 || hb[3 * i] < -1e-12 || hb[3 * i + 1] < -1e-12 ||
            hb[3 * i + 2] < -1e-12) {
            c->err = "particles_set: barycentric triple must be finite, >= 0 and sum to 1";
            return CSS_ERR_INVALID_ARG;
        }
    }
    css_parts* p = new css_parts();
    p->ctx = c;
    p->mesh = m;
    p->n = n;
    p->seed = seed;
    cudaStream_t st = c->stream;
    cudaError_t e = cudaSuccess;
    const size_t nf = (size_t)m->nf;
    // one contiguous block: bary | vel | orient | force | face, so a snapshot is one copy
    e = cudaMalloc(&p->state, p->state_bytes());
    if (e == cudaSuccess) {
        p->bary = (double*)p->state;
        p->vel = p->bary + 3 * n;
        p->orient = p->bary + 6 * n;
        p->force = p->bary + 9 * n;
        p->face = (int32_t*)(p->bary + 12 * n);
        e = cudaMemcpyAsync(p->face, hf.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->bary, hb.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMalloc(&p->fcnt, (nf + 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->fstart, (nf + 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->fitems, n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->scan_tmp, cssi::scan_tmp_ints(nf + 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->pcnt, n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->dstep, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->dstep, 0, sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->fcnt, 0, (nf + 1) * sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->force, 0, 3 * n * sizeof(double), st);
    if (e == cudaSuccess) e = vel ? cudaMemcpyAsync(p->vel, vel, 3 * n * sizeof(double), is_device_ptr(vel) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st)
                                  : cudaMemsetAsync(p->vel, 0, 3 * n * sizeof(double), st);
    if (e == cudaSuccess) e = orient ? cudaMemcpyAsync(p->orient, orient, 3 * n * sizeof(double), is_device_ptr(orient) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st)
                                     : cudaMemsetAsync(p->orient, 0, 3 * n * sizeof(double), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { css_particles_free(p); return cuda_fail(c, "particles_set", e); }
    *out = p;
    return CSS_OK;
}

int css_particles_get(css_parts* p, int32_t* face, double* bary, double* vel, double* orient, double* force,
                      int64_t* step) {
    if (!p) return CSS_ERR_INVALID_ARG;
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    TRY(c, "particles_get", copy_out(face, p->face, p->n, st));
    TRY(c, "particles_get", copy_out(bary, p->bary, 3 * p->n, st));
    TRY(c, "particles_get", copy_out(vel, p->vel, 3 * p->n, st));
    TRY(c, "particles_get", copy_out(orient, p->orient, 3 * p->n, st));
    TRY(c, "particles_get", copy_out(force, p->force, 3 * p->n, st));
    TRY(c, "particles_get", cudaStreamSynchronize(st));
    if (step) *step = p->step;
    return CSS_OK;
}

int css_particles_update(css_parts* p, const int32_t* face, const double* bary, const double* vel,
                         const double* orient) {
    if (!p) return CSS_ERR_INVALID_ARG;
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    auto kind = [](const void* q) { return is_device_ptr(q) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; };
    if (face) {
        if (!is_device_ptr(face))
            for (int64_t i = 0; i < p->n; ++i)
                if (face[i] < 0 || face[i] >= p->mesh->nf) { c->err = "particles_update: face index out of range"; return CSS_ERR_INVALID_ARG; }
        TRY(c, "particles_update", cudaMemcpyAsync(p->face, face, p->n * sizeof(int32_t), kind(face), st));
    }
    if (bary) TRY(c, "particles_update", cudaMemcpyAsync(p->bary, bary, 3 * p->n * sizeof(double), kind(bary), st));
    if (vel) TRY(c, "particles_update", cudaMemcpyAsync(p->vel, vel, 3 * p->n * sizeof(double), kind(vel), st));
    if (orient) TRY(c, "particles_update", cudaMemcpyAsync(p->orient, orient, 3 * p->n * sizeof(double), kind(orient), st));
    if (face || bary) p->force_valid = 0;
    return CSS_OK;
}

int css_particles_free(css_parts* p) {
    if (!p) return CSS_ERR_INVALID_ARG;
    if (p->graph) cudaGraphExecDestroy(p->graph);
    cudaFree(p->state); cudaFree(p->snap);
    cudaFree(p->fcnt); cudaFree(p->fstart); cudaFree(p->fitems); cudaFree(p->scan_tmp); cudaFree(p->order);
    cudaFree(p->pcnt); cudaFree(p->pj); cudaFree(p->pd); cudaFree(p->pt); cudaFree(p->dstep);
    delete p;
    return CSS_OK;
}


int css_geodesic_neighbors(css_parts* p, double r_c, int precision, int64_t capacity, int64_t* n_pairs,
                           int64_t* row_start, int32_t* nbr_j, double* dist, double* tangent) {
    if (!p || !n_pairs || bad_prec(precision) || bad_rc(r_c) || capacity < 0) return CSS_ERR_INVALID_ARG;
    css_ctx* c = p->ctx;
    int rc = run_geo(p, r_c, precision, 1, 0, nullptr);
    if (rc) return rc;
    cudaStream_t st = c->stream;
    const int32_t n = (int32_t)p->n;
    int64_t* drows = nullptr;
    TRY(c, "neighbors", cudaMalloc(&drows, (n + 1 + cssi::scan_tmp_ints(n + 1)) * sizeof(int64_t)));
    cudaError_t e = cssi::launch_scan_rows(p->pcnt, drows, n, st);
    int64_t total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, drows + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFree(drows); return cuda_fail(c, "neighbors", e); }
    *n_pairs = total;
    if (total > capacity) { cudaFree(drows); c->err = "neighbors: capacity too small"; return CSS_ERR_CAPACITY; }
    if (!row_start || (total > 0 && (!nbr_j || !dist || !tangent))) { cudaFree(drows); return CSS_ERR_INVALID_ARG; }
    const bool dev_out = is_device_ptr(nbr_j) && is_device_ptr(dist) && is_device_ptr(tangent);
    int32_t* oj = nbr_j;
    double* od = dist;
    double* ot = tangent;
    if (!dev_out && total > 0) {
        e = cudaMalloc(&oj, total * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&od, total * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&ot, 3 * total * sizeof(double));
        if (e != cudaSuccess) { cudaFree(drows); return cuda_fail(c, "neighbors", e); }
    }
    if (total > 0) e = cssi::launch_pairs_compact(n, p->pcnt, p->pj, p->pd, p->pt, p->pair_cap_alloc, drows, oj, od, ot, st);
    if (e == cudaSuccess) e = copy_out(row_start, drows, (size_t)n + 1, st);
    if (!dev_out && total > 0) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(nbr_j, oj, total * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dist, od, total * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tangent, ot, 3 * total * sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (!dev_out && total > 0) { cudaFree(oj); cudaFree(od); cudaFree(ot); }
    cudaFree(drows);
    if (e != cudaSuccess) return cuda_fail(c, "neighbors", e);
    return CSS_OK;
}

int css_compute_forces(css_parts* p, const css_potential* pot, double r_c, int precision, double* forces, double* e_pot) {
    if (!p || !pot || bad_prec(precision) || bad_rc(r_c) || pot->kind < 0 || pot->kind > 2) return CSS_ERR_INVALID_ARG;
    css_ctx* c = p->ctx;
    int rc = run_geo(p, r_c, precision, 0, 1, pot);
    if (rc) return rc;
    p->force_valid = 1;
    p->force_rc = r_c;
    p->force_prec = precision;
    p->force_pot = *pot;
    TRY(c, "forces", copy_out(forces, p->force, 3 * p->n, c->stream));
    if (e_pot) TRY(c, "forces", cudaMemcpyAsync(e_pot, c->depot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TRY(c, "forces", cudaStreamSynchronize(c->stream));
    return CSS_OK;
}

// ------------------------------------------------------------------------------ stepping
namespace {

cudaError_t snap_take(css_parts* p) {
    if (!p->snap) {
        cudaError_t e = cudaMalloc(&p->snap, p->state_bytes());
        if (e != cudaSuccess) return e;
    }
    return cudaMemcpyAsync(p->snap, p->state, p->state_bytes(), cudaMemcpyDeviceToDevice, p->ctx->stream);
}

cudaError_t snap_restore(css_parts* p) {
    cudaStream_t st = p->ctx->stream;
    cudaError_t e = cudaMemcpyAsync(p->state, p->snap, p->state_bytes(), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(p->dstep, &p->step, sizeof(int64_t), cudaMemcpyHostToDevice, st);
}

// per-set integrator kernels of one step: NVE half = 0 before the forces (kick + drift),
// half = 1 after them (kick); overdamped dynamics move after the forces
int enqueue_move(css_parts* p, const css_integrator* it, const double* noise, int half) {
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    const int32_t n = (int32_t)p->n;
    if (it->kind == CSS_INT_NVE) {
        if (half == 0)
            TRY(c, "kick_drift", cssi::launch_nve_kick_drift(p->mesh->view(), n, p->face, p->bary, p->vel, p->force, *it,
                                                             c->dscal + 1, st));
        else
            TRY(c, "kick", cssi::launch_nve_kick(n, p->vel, p->force, *it, st));
    } else if (half == 1) {
        TRY(c, "move", cssi::launch_overdamped_move(p->mesh->view(), n, p->face, p->bary, p->orient, p->force, *it,
                                                    p->seed, p->dstep, noise, c->dscal + 1, st));
        TRY(c, "step", cssi::launch_step_inc(p->dstep, st));
    }
    return CSS_OK;
}

// enqueue one full step (no synchronisation); noise: device pointer to n x 2 normals or NULL
int enqueue_step(css_parts* p, const css_potential* pot, const css_integrator* it, double rc, int prec,
                 const double* noise, const GeoWs& g, int nctas) {
    css_ctx* c = p->ctx;
    int r = enqueue_move(p, it, noise, 0);
    if (r) return r;
    TRY(c, "reset", cudaMemsetAsync(c->depot, 0, sizeof(double), c->stream));
    r = enqueue_geo(p, rc, prec, 0, 1, pot, g, nctas);
    if (r) return r;
    return enqueue_move(p, it, noise, 1);
}

// capture fn() on the context stream into an executable graph
template <class Fn>
int capture(css_ctx* c, Fn fn, cudaGraphExec_t* exec) {
    cudaStream_t st = c->stream;
    cudaGraph_t graph = nullptr;
    TRY(c, "capture", cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = fn();
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return cuda_fail(c, "capture", e);
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c, "graph instantiate", e);
    return CSS_OK;
}

}  // namespace

int css_integrate_step(css_parts* p, const css_potential* pot, const css_integrator* it, double r_c, int precision,
                       int64_t n_steps, const double* noise, double* e_pot) {
    if (!p || !pot || !it || bad_prec(precision) || bad_rc(r_c) || n_steps < 0 || it->kind < 0 || it->kind > 2 ||
        !(it->dt > 0.0) || !(it->mass > 0.0) || !(it->lambda > 0.0) || !(it->max_disp > 0.0))
        return CSS_ERR_INVALID_ARG;
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    if (n_steps == 0) return CSS_OK;
    // NVE needs the force at the current positions
    if (it->kind == CSS_INT_NVE &&
        !(p->force_valid && p->force_rc == r_c && p->force_prec == precision &&
          memcmp(&p->force_pot, pot, sizeof(css_potential)) == 0)) {
        int rc = css_compute_forces(p, pot, r_c, precision, nullptr, nullptr);
        if (rc) return rc;
    }
    double* dnoise = nullptr;
    if (noise) {
        const size_t cnt = (size_t)n_steps * p->n * 2;
        if (is_device_ptr(noise)) dnoise = const_cast<double*>(noise);
        else {
            TRY(c, "noise", cudaMalloc(&dnoise, cnt * sizeof(double)));
            TRY(c, "noise", cudaMemcpyAsync(dnoise, noise, cnt * sizeof(double), cudaMemcpyHostToDevice, st));
        }
    }
    int retries = 0;
    int rc = CSS_OK;
    for (;;) {
        TRY(c, "snapshot", snap_take(p));
        GeoWs g;
        int nctas = 0;
        const int shared = use_shared(p);
        rc = ensure_ws(c, precision, shared, &g, &nctas);
        if (rc) break;
        TRY(c, "reset", cudaMemsetAsync(c->dscal + 1, 0, sizeof(int), st));
        TRY(c, "reset", cudaMemsetAsync(c->dcount, 0, 8 * sizeof(unsigned long long), st));
        if (!dnoise) {
            // one captured step, kept with the parameters it was captured for, replayed
            std::string key((const char*)pot, sizeof(*pot));
            key.append((const char*)it, sizeof(*it));
            key.append((const char*)&r_c, sizeof(r_c));
            const int64_t shape[5] = {precision, c->ws_key, nctas, (int64_t)(uintptr_t)c->ws, shared};
            key.append((const char*)shape, sizeof(shape));
            if (!p->graph || p->graph_key != key) {
                if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
                rc = capture(c, [&]() { return enqueue_step(p, pot, it, r_c, precision, nullptr, g, nctas); }, &p->graph);
                if (rc == CSS_OK) p->graph_key = key;
            }
            for (int64_t s = 0; s < n_steps && rc == CSS_OK; ++s) {
                cudaError_t e = cudaGraphLaunch(p->graph, st);
                if (e != cudaSuccess) rc = cuda_fail(c, "graph launch", e);
            }
        } else {
            for (int64_t s = 0; s < n_steps && rc == CSS_OK; ++s)
                rc = enqueue_step(p, pot, it, r_c, precision, dnoise ? dnoise + (size_t)s * p->n * 2 : nullptr, g, nctas);
        }
        if (rc) break;
        int status = 0;
        rc = read_status(c, &status);
        if (rc) break;
        if (status == 0) break;
        bool to_global = false;
        if (!grow_for(c, status, &retries, shared, &to_global)) { rc = status_error(c, status); break; }
        if (to_global) p->global_tables = 1;
        TRY(c, "restore", snap_restore(p));
    }
    if (noise && !is_device_ptr(noise)) cudaFree(dnoise);
    if (rc) return rc;
    p->step += n_steps;
    p->force_valid = 1;
    p->force_rc = r_c;
    p->force_prec = precision;
    p->force_pot = *pot;
    if (e_pot) {
        TRY(c, "e_pot", cudaMemcpyAsync(e_pot, c->depot, sizeof(double), cudaMemcpyDeviceToHost, st));
        TRY(c, "e_pot", cudaStreamSynchronize(st));
    }
    return CSS_OK;
}

// ------------------------------------------------------------------------------ batched form
struct css_batch {
    css_ctx* ctx = nullptr;
    std::vector<css_parts*> sets;
    GeoJob* djobs = nullptr;
    int32_t* job_of_item = nullptr;
    int32_t* src_of_item = nullptr;
    int32_t nitems = 0;
};

int css_batch_create(css_ctx* c, css_parts* const* parts, int32_t n_sets, css_batch** out) {
    if (!c || !parts || !out || n_sets < 1) return CSS_ERR_INVALID_ARG;
    *out = nullptr;
    css_batch* b = new css_batch();
    b->ctx = c;
    int64_t total = 0;
    for (int k = 0; k < n_sets; ++k) {
        if (!parts[k] || parts[k]->ctx != c) { delete b; return CSS_ERR_INVALID_ARG; }
        b->sets.push_back(parts[k]);
        total += parts[k]->n;
    }
    if (total > INT32_MAX) { delete b; return CSS_ERR_INVALID_ARG; }
    // work items ordered by set size (largest first): a crude cost proxy refined by the
    // caller's autotuning of the launch shape
    std::vector<int> ord(n_sets);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int bb) { return b->sets[a]->n > b->sets[bb]->n; });
    std::vector<int32_t> hj, hs;
    hj.reserve(total);
    hs.reserve(total);
    for (int k : ord)
        for (int64_t i = 0; i < b->sets[k]->n; ++i) { hj.push_back(k); hs.push_back((int32_t)i); }
    b->nitems = (int32_t)total;
    cudaError_t e = cudaMalloc(&b->djobs, n_sets * sizeof(GeoJob));
    if (e == cudaSuccess) e = stage_in(hj.data(), hj.size(), &b->job_of_item, c->stream);
    if (e == cudaSuccess) e = stage_in(hs.data(), hs.size(), &b->src_of_item, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { css_batch_free(b); return cuda_fail(c, "batch_create", e); }
    *out = b;
    return CSS_OK;
}

int css_batch_free(css_batch* b) {
    if (!b) return CSS_ERR_INVALID_ARG;
    cudaFree(b->djobs);
    cudaFree(b->job_of_item);
    cudaFree(b->src_of_item);
    delete b;
    return CSS_OK;
}

namespace {

int batch_enqueue_forces(css_batch* b, const css_potential* pot, double rc, int prec, const GeoWs& g, int nctas) {
    css_ctx* c = b->ctx;
    cudaStream_t st = c->stream;
    for (css_parts* p : b->sets)
        TRY(c, "bucket", cssi::launch_bucket((int32_t)p->n, (int32_t)p->mesh->nf, p->face, p->fcnt, p->fstart,
                                             p->fitems, p->scan_tmp, st));
    TRY(c, "reset", cudaMemsetAsync(c->dscal, 0, sizeof(int), st));
    TRY(c, "reset", cudaMemsetAsync(c->depot, 0, sizeof(double), st));
    GeoJob j0 = make_job(b->sets[0], rc, 0, 1, pot);
    TRY(c, "event", record_ev(c, c->ev_geo0));
    TRY(c, "geodesic", cssi::launch_geodesic(j0, b->djobs, b->job_of_item, b->src_of_item, b->nitems, prec, g,
                                             c->warps_per_cta, nctas, c->dscal, c->dscal + 1, c->dcount, st));
    TRY(c, "event", record_ev(c, c->ev_geo1));
    return CSS_OK;
}

}  // namespace

int css_batch_step(css_batch* b, const css_potential* pot, const css_integrator* it, double r_c, int precision,
                   int64_t n_steps) {
    if (!b || !pot || !it || bad_prec(precision) || bad_rc(r_c) || n_steps < 0 || it->kind < 0 || it->kind > 2 ||
        !(it->dt > 0.0) || !(it->mass > 0.0) || !(it->lambda > 0.0) || !(it->max_disp > 0.0))
        return CSS_ERR_INVALID_ARG;
    css_ctx* c = b->ctx;
    cudaStream_t st = c->stream;
    if (n_steps == 0) return CSS_OK;
    {   // device copy of the per-set job descriptors
        std::vector<GeoJob> hj;
        for (css_parts* p : b->sets) hj.push_back(make_job(p, r_c, 0, 1, pot));
        TRY(c, "batch jobs", cudaMemcpyAsync(b->djobs, hj.data(), hj.size() * sizeof(GeoJob), cudaMemcpyHostToDevice, st));
        TRY(c, "batch jobs", cudaStreamSynchronize(st));
    }
    // NVE needs the forces at the starting positions unless every set still holds them
    bool nve = it->kind == CSS_INT_NVE;
    if (nve) {
        bool valid = true;
        for (css_parts* p : b->sets)
            valid = valid && p->force_valid && p->force_rc == r_c && p->force_prec == precision &&
                    memcmp(&p->force_pot, pot, sizeof(css_potential)) == 0;
        nve = !valid;
    }
    int retries = 0;
    for (;;) {
        for (css_parts* p : b->sets) TRY(c, "snapshot", snap_take(p));
        GeoWs g;
        int nctas = 0;
        int shared = c->shared_tables;
        for (css_parts* p : b->sets) shared = shared && !p->global_tables;
        int rc = ensure_ws(c, precision, shared, &g, &nctas);
        if (rc) return rc;
        TRY(c, "reset", cudaMemsetAsync(c->dscal + 1, 0, sizeof(int), st));
        TRY(c, "reset", cudaMemsetAsync(c->dcount, 0, 8 * sizeof(unsigned long long), st));
        if (nve) {   // forces at the starting positions
            rc = batch_enqueue_forces(b, pot, r_c, precision, g, nctas);
            if (rc) return rc;
        }
        auto one_step = [&]() -> int {
            for (css_parts* p : b->sets) { int r = enqueue_move(p, it, nullptr, 0); if (r) return r; }
            int r = batch_enqueue_forces(b, pot, r_c, precision, g, nctas);
            if (r) return r;
            for (css_parts* p : b->sets) { r = enqueue_move(p, it, nullptr, 1); if (r) return r; }
            return CSS_OK;
        };
        cudaGraphExec_t exec = nullptr;
        rc = capture(c, one_step, &exec);
        for (int64_t s = 0; s < n_steps && rc == CSS_OK; ++s) {
            cudaError_t e = cudaGraphLaunch(exec, st);
            if (e != cudaSuccess) rc = cuda_fail(c, "graph launch", e);
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (rc) return rc;
        int status = 0;
        rc = read_status(c, &status);
        if (rc) return rc;
        if (status == 0) break;
        bool to_global = false;
        if (!grow_for(c, status, &retries, shared, &to_global)) return status_error(c, status);
        if (to_global) for (css_parts* p : b->sets) p->global_tables = 1;
        for (css_parts* p : b->sets) TRY(c, "restore", snap_restore(p));
    }
    for (css_parts* p : b->sets) {
        p->step += n_steps;
        p->force_valid = 1;
        p->force_rc = r_c;
        p->force_prec = precision;
        p->force_pot = *pot;
    }
    return CSS_OK;
}

