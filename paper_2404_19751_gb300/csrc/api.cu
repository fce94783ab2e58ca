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

#include <nvtx3/nvToolsExt.h>

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

// ---- workspaces of the two passes of the persistent neighbour/force kernel
struct GeoPlan {
    GeoWs g1, g2;
    int wpc1 = 0, nctas1 = 0, wpc2 = 0, nctas2 = 0;
    int team = 0;   // first pass in the team form (one source per CTA)
};

// size (and zero on a layout change, so old bytes never look like valid hash tags) one
// pass's workspace
int ensure_buf(css_ctx* c, cssi::WsBuf& b, int precision, int win_cap, int tab_cap, int shared, int nwarps,
               GeoWs* out) {
    GeoWs g{};
    g.shared = shared;
    g.stride = cssi::geo_ws_bytes_per_warp(precision, win_cap, shared ? 0 : tab_cap, &g.log_eh, &g.log_vh, &g.log_fh,
                                           &g.fcap, &g.emcap);
    g.wcap = win_cap;
    g.nwarps = nwarps;
    const size_t need = g.stride * (size_t)nwarps;
    const int64_t key = (((int64_t)precision * 1000003 + (int64_t)win_cap * 31 + nwarps) * 16 + shared) * 2097152 +
                        (shared ? 0 : tab_cap);
    const bool relayout = (need > b.bytes) || (b.warps < nwarps) || (b.key != key);
    if (need > b.bytes) {
        cudaFree(b.ws);
        b.ws = nullptr;
        b.bytes = 0;
        TRY(c, "workspace", cudaMalloc(&b.ws, need));
        b.bytes = need;
    }
    if (b.warps < nwarps) {
        cudaFree(b.gen);
        b.gen = nullptr;
        TRY(c, "workspace", cudaMalloc(&b.gen, nwarps * sizeof(uint32_t)));
        b.warps = nwarps;
    }
    if (relayout) {
        TRY(c, "workspace", cudaMemsetAsync(b.ws, 0, b.bytes, c->stream));
        TRY(c, "workspace", cudaMemsetAsync(b.gen, 0, b.warps * sizeof(uint32_t), c->stream));
        b.key = key;
    }
    g.base = (char*)b.ws;
    g.gen = b.gen;
    *out = g;
    return CSS_OK;
}

// both passes for the context's launch shape and up to `nitems` work items
int ensure_plan(css_ctx* c, int precision, int64_t nitems, GeoPlan* P) {
    const cssi::LaunchCfg& L = c->cfg;
    // the occupancy query costs host time on every call: cached per shape
    const int64_t bkey = (((int64_t)precision * 64 + L.warps_per_cta) * 64 + L.shared_scale * 4 + L.occupancy) * 2 + L.team;
    auto hit = c->bps_cache.find(bkey);
    int bps = hit != c->bps_cache.end()
                  ? hit->second
                  : (c->bps_cache[bkey] = L.team ? cssi::geodesic_team_blocks_per_sm(precision, L.warps_per_cta,
                                                                                     L.shared_scale, L.occupancy)
                                                 : cssi::geodesic_blocks_per_sm(precision, L.warps_per_cta,
                                                                                L.shared_scale, L.occupancy));
    if (bps < 1) {
        c->err = "launch shape does not fit an SM (" + std::to_string(L.warps_per_cta) + " warps per CTA, shared scale " +
                 std::to_string(L.shared_scale) + ")";
        return CSS_ERR_INVALID_ARG;
    }
    if (L.ctas_per_sm > 0) bps = std::min(bps, L.ctas_per_sm);
    P->wpc1 = L.warps_per_cta;
    P->nctas1 = c->sm_count * bps;
    P->team = L.team;
    // one workspace slice per warp, or per CTA in the team form
    int rc = ensure_buf(c, c->ws1, precision, L.win_cap, L.tab_cap, L.shared_scale,
                        L.team ? P->nctas1 : P->nctas1 * P->wpc1, &P->g1);
    if (rc) return rc;
    P->g1.occupancy = L.occupancy;
    P->wpc2 = L.warps2_per_sm;
    P->nctas2 = c->sm_count;
    rc = ensure_buf(c, c->ws2, precision, L.win_cap2, 0, 0, P->nctas2 * P->wpc2, &P->g2);
    if (rc) return rc;
    P->g2.occupancy = 1;
    if (c->defer_cap < nitems) {
        cudaFree(c->defer);
        c->defer = nullptr;
        c->defer_cap = 0;
        TRY(c, "deferral list", cudaMalloc(&c->defer, std::max<int64_t>(nitems, 1) * sizeof(int32_t)));
        c->defer_cap = nitems;
    }
    return CSS_OK;
}

// the plan's identity, for keying captured graphs
std::string plan_key(const css_ctx* c, const GeoPlan& P) {
    const int64_t v[8] = {c->ws1.key, c->ws2.key, (int64_t)(uintptr_t)c->ws1.ws, (int64_t)(uintptr_t)c->ws2.ws,
                          (int64_t)(uintptr_t)c->defer, P.nctas1, (c->cfg.tile * 8 + c->cfg.occupancy) * 2 + P.team,
                          P.nctas2};
    return std::string((const char*)v, sizeof(v));
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
    j.order = p->fitems;   // sources in face-rank (Morton) order
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

// the two passes over a work queue, timed by the context's events (no synchronisation)
int enqueue_passes(css_ctx* c, const GeoJob& j0, const GeoJob* djobs, const int32_t* job_of_item,
                   const int32_t* src_of_item, int32_t nitems, int prec, const GeoPlan& P) {
    cudaStream_t st = c->stream;
    TRY(c, "reset", cudaMemsetAsync(c->dscal, 0, sizeof(int), st));
    TRY(c, "reset", cudaMemsetAsync(c->dscal + 2, 0, 2 * sizeof(int), st));
    TRY(c, "event", record_ev(c, c->ev_geo0));
    cssi::GeoQueue q1{job_of_item, src_of_item, nitems, nullptr, nullptr, c->defer, c->dscal + 2, c->cfg.tile};
    if (P.team)
        TRY(c, "geodesic", cssi::launch_geodesic_team(j0, djobs, q1, prec, P.g1, P.wpc1, P.nctas1, c->dscal,
                                                      c->dscal + 1, c->dcount, st));
    else
        TRY(c, "geodesic", cssi::launch_geodesic(j0, djobs, q1, prec, P.g1, P.wpc1, P.nctas1, c->dscal, c->dscal + 1,
                                                 c->dcount, st));
    cssi::GeoQueue q2{job_of_item, src_of_item, nitems, c->defer, c->dscal + 2, nullptr, nullptr, 1};
    TRY(c, "geodesic", cssi::launch_geodesic(j0, djobs, q2, prec, P.g2, P.wpc2, P.nctas2, c->dscal + 3, c->dscal + 1,
                                             c->dcount, st));
    TRY(c, "event", record_ev(c, c->ev_geo1));
    return CSS_OK;
}

// one bucket + neighbour/force evaluation of one set (no synchronisation)
int enqueue_geo(css_parts* p, double rc, int prec, int want_pairs, int want_forces, const css_potential* pot,
                const GeoPlan& P) {
    css_ctx* c = p->ctx;
    TRY(c, "bucket", cssi::launch_bucket((int32_t)p->n, (int32_t)p->mesh->nf, p->face, p->mesh->frank, p->fcnt, p->fstart, p->fitems, p->ftmp,
                                         p->scan_tmp, c->stream));
    GeoJob j = make_job(p, rc, want_pairs, want_forces, pot);
    return enqueue_passes(c, j, nullptr, nullptr, nullptr, (int32_t)p->n, prec, P);
}

int read_status(css_ctx* c, int* status) {
    TRY(c, "status", cudaMemcpyAsync(c->hstat, c->dscal + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    TRY(c, "status", cudaMemcpyAsync(c->hcount, c->dcount, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    TRY(c, "sync", cudaStreamSynchronize(c->stream));
    *status = *c->hstat;
    for (int k = 0; k < 5; ++k) c->last_counters[k] = (int64_t)c->hcount[k];
    return CSS_OK;
}

// grow the capacity that overflowed in the second pass (the first pass defers instead of
// failing); false when nothing can grow any more
bool grow_for(css_ctx* c, int status, int* retries) {
    ++*retries;
    ++c->last_counters[5];
    if (*retries > MAX_RETRY) return false;
    bool grown = false;
    if (status & (css::ST_WIN_OVERFLOW | css::ST_HASH_OVERFLOW | css::ST_ITER_LIMIT)) {
        if (c->cfg.win_cap2 >= WIN_CAP_MAX) return false;
        c->cfg.win_cap2 *= 2;
        grown = true;
    }
    if (status & css::ST_PAIR_OVERFLOW) { c->pair_cap *= 2; grown = true; }
    return grown;
}

int status_error(css_ctx* c, int status) {
    if (status & (css::ST_WIN_OVERFLOW | css::ST_HASH_OVERFLOW)) {
        c->err = "window workspace exhausted (capacity " + std::to_string(c->cfg.win_cap2) + ")";
        return CSS_ERR_QUEUE_OVERFLOW;
    }
    if (status & (css::ST_ITER_LIMIT | css::ST_WALK_LIMIT)) { c->err = "device loop reached its iteration cap"; return CSS_ERR_ITER_LIMIT; }
    if (status & css::ST_PIECES) { c->err = "window trimming produced too many pieces"; return CSS_ERR_QUEUE_OVERFLOW; }
    if (status & css::ST_PAIR_OVERFLOW) { c->err = "pair slab overflow"; return CSS_ERR_QUEUE_OVERFLOW; }
    c->err = "device status " + std::to_string(status);
    return CSS_ERR_CUDA;
}

// A context whose launch shape nobody set or tuned adapts its first pass: when more than a
// quarter of the evaluated sources were deferred (patches too large for the shared tables
// or the pool), later evaluations use global tables and a four times larger pool.
void adapt_default(css_ctx* c) {
    if (c->cfg_explicit) return;
    const int64_t done = c->last_counters[0], deferred = c->last_counters[4];
    if (done > 0 && deferred * 4 > done && c->cfg.win_cap < (1 << 17)) {
        c->cfg.shared_scale = 0;
        c->cfg.win_cap = std::max(c->cfg.win_cap * 4, 8192);
    }
}

// synchronous neighbour / force evaluation with overflow retries
int run_geo(css_parts* p, double rc, int prec, int want_pairs, int want_forces, const css_potential* pot) {
    css_ctx* c = p->ctx;
    int retries = 0;
    c->last_counters[5] = 0;
    for (;;) {
        if (want_pairs) { int rc2 = ensure_pairs(p, c->pair_cap); if (rc2) return rc2; }
        GeoPlan P;
        int rc1 = ensure_plan(c, prec, p->n, &P);
        if (rc1) return rc1;
        TRY(c, "reset", cudaMemsetAsync(c->dcount, 0, 8 * sizeof(unsigned long long), c->stream));
        TRY(c, "reset", cudaMemsetAsync(c->dscal + 1, 0, sizeof(int), c->stream));
        TRY(c, "reset", cudaMemsetAsync(c->depot, 0, sizeof(double), c->stream));
        rc1 = enqueue_geo(p, rc, prec, want_pairs, want_forces, pot, P);
        if (rc1) return rc1;
        int status = 0;
        rc1 = read_status(c, &status);
        if (rc1) return rc1;
        if (status == 0) { adapt_default(c); return CSS_OK; }
        if (!grow_for(c, status, &retries)) return status_error(c, status);
    }
}

bool finite_all(const double* h, size_t n) {
    for (size_t i = 0; i < n; ++i) if (!std::isfinite(h[i])) return false;
    return true;
}

}  // namespace

namespace {
// one NVTX range per public call that launches work (visible to profilers and tracers;
// free when no tool is attached)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};
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
    if (cudaEventCreate(&c->ev_geo0) != cudaSuccess || cudaEventCreate(&c->ev_geo1) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_order, cudaEventDisableTiming) != cudaSuccess) {
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
    cudaFree(c->ws1.ws);
    cudaFree(c->ws1.gen);
    cudaFree(c->ws2.ws);
    cudaFree(c->ws2.gen);
    cudaFree(c->defer);
    cudaFree(c->dscal);
    cudaFree(c->dcount);
    cudaFree(c->depot);
    cudaFreeHost(c->hstat);
    cudaFreeHost(c->hcount);
    if (c->ev_geo0) cudaEventDestroy(c->ev_geo0);
    if (c->ev_geo1) cudaEventDestroy(c->ev_geo1);
    if (c->ev_order) cudaEventDestroy(c->ev_order);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return CSS_OK;
}

const char* css_last_error(const css_ctx* c) { return c ? c->err.c_str() : "null context"; }

int css_last_counters(const css_ctx* c, int64_t out[6]) {
    if (!c || !out) return CSS_ERR_INVALID_ARG;
    for (int k = 0; k < 6; ++k) out[k] = c->last_counters[k];
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

static bool launch_ok(const css_launch* l) {
    const int s = l->shared_scale;
    return l->warps_per_cta >= 1 && l->warps_per_cta <= 8 && l->ctas_per_sm >= 0 && l->ctas_per_sm <= 32 &&
           l->tile >= 1 && l->tile <= 64 && (s == 0 || s == 1 || s == 2 || s == 4 || s == 8) &&
           l->window_capacity >= 64 && l->window_capacity <= (1 << 20) && l->window_capacity2 >= 64 &&
           l->window_capacity2 <= (1 << 20) && l->warps2_per_sm >= 1 && l->warps2_per_sm <= 8 &&
           (l->occupancy == 1 || l->occupancy == 2) &&
           (l->table_capacity == 0 || (l->table_capacity >= 64 && l->table_capacity <= (1 << 20))) &&
           (l->team == 0 || (l->team == 1 && l->warps_per_cta >= 2));
}

int css_set_launch(css_ctx* c, const css_launch* l) {
    if (!c || !l || !launch_ok(l)) return CSS_ERR_INVALID_ARG;
    for (int prec : {CSS_FP32, CSS_FP64})
        if ((l->team ? cssi::geodesic_team_blocks_per_sm(prec, l->warps_per_cta, l->shared_scale, l->occupancy)
                     : cssi::geodesic_blocks_per_sm(prec, l->warps_per_cta, l->shared_scale, l->occupancy)) < 1) {
            c->err = "launch shape does not fit an SM";
            return CSS_ERR_INVALID_ARG;
        }
    c->cfg.warps_per_cta = l->warps_per_cta;
    c->cfg.ctas_per_sm = l->ctas_per_sm;
    c->cfg.tile = l->tile;
    c->cfg.shared_scale = l->shared_scale;
    c->cfg.win_cap = next_pow2(l->window_capacity);
    c->cfg.win_cap2 = next_pow2(l->window_capacity2);
    c->cfg.warps2_per_sm = l->warps2_per_sm;
    c->cfg.occupancy = l->occupancy;
    c->cfg.tab_cap = l->table_capacity ? next_pow2(l->table_capacity) : 0;
    c->cfg.team = l->team;
    c->cfg_explicit = 1;
    return CSS_OK;
}

int css_get_launch(const css_ctx* c, css_launch* l) {
    if (!c || !l) return CSS_ERR_INVALID_ARG;
    l->warps_per_cta = c->cfg.warps_per_cta;
    l->ctas_per_sm = c->cfg.ctas_per_sm;
    l->tile = c->cfg.tile;
    l->shared_scale = c->cfg.shared_scale;
    l->window_capacity = c->cfg.win_cap;
    l->window_capacity2 = c->cfg.win_cap2;
    l->warps2_per_sm = c->cfg.warps2_per_sm;
    l->occupancy = c->cfg.occupancy;
    l->table_capacity = c->cfg.tab_cap;
    l->team = c->cfg.team;
    return CSS_OK;
}

int css_mesh_upload(css_ctx* c, const double* verts, int64_t nv, const int32_t* faces, int64_t nf, const double* period,
                    css_mesh** out) {
    Range range_("css_mesh_upload");
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
    cudaFree(m->frank);
    cudaFree(m->cang);
    cssi::vhm_free(m);
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
    Range range_("css_particles_set");
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
    if (e == cudaSuccess) e = cudaMalloc(&p->ftmp, n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->scan_tmp, cssi::scan_tmp_ints(nf + 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->pcnt, n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->dstep, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->dfire, 16 * sizeof(double));
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
    Range range_("css_particles_update");
    if (!p) return CSS_ERR_INVALID_ARG;
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    auto kind = [](const void* q) { return is_device_ptr(q) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; };
    if ((face || bary || vel) && (p->force_valid || p->fire_valid)) {
        // forces (or a FIRE state) are cached for the current state: stage the upload in the
        // snapshot buffer, compare it bitwise with the current state, then copy it in; an
        // upload of an unchanged state (a host loop that writes back what it read) keeps them
        if (face && !is_device_ptr(face))
            for (int64_t i = 0; i < p->n; ++i)
                if (face[i] < 0 || face[i] >= p->mesh->nf) { c->err = "particles_update: face index out of range"; return CSS_ERR_INVALID_ARG; }
        if (!p->snap) TRY(c, "particles_update", cudaMalloc(&p->snap, p->state_bytes()));
        const int64_t n = p->n;
        double* sb = (double*)p->snap;                 // same layout as the state block
        double* sv = sb + 3 * n;
        int32_t* sf = (int32_t*)(sb + 12 * n);
        if (face) TRY(c, "particles_update", cudaMemcpyAsync(sf, face, n * sizeof(int32_t), kind(face), st));
        if (bary) TRY(c, "particles_update", cudaMemcpyAsync(sb, bary, 3 * n * sizeof(double), kind(bary), st));
        if (vel) TRY(c, "particles_update", cudaMemcpyAsync(sv, vel, 3 * n * sizeof(double), kind(vel), st));
        TRY(c, "particles_update", cudaMemsetAsync(c->dscal + 1, 0, sizeof(int), st));
        TRY(c, "particles_update", cssi::launch_state_diff((int32_t)n, face ? sf : nullptr, p->face, bary ? sb : nullptr,
                                                           p->bary, vel ? sv : nullptr, p->vel, c->dscal + 1, st));
        if (face) TRY(c, "particles_update", cudaMemcpyAsync(p->face, sf, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        if (bary) TRY(c, "particles_update", cudaMemcpyAsync(p->bary, sb, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (vel) TRY(c, "particles_update", cudaMemcpyAsync(p->vel, sv, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (orient) TRY(c, "particles_update", cudaMemcpyAsync(p->orient, orient, 3 * n * sizeof(double), kind(orient), st));
        TRY(c, "particles_update", cudaMemcpyAsync(c->hstat, c->dscal + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        TRY(c, "particles_update", cudaStreamSynchronize(st));
        const int changed = *c->hstat;
        if (changed & 1) p->force_valid = 0;
        if (changed & 3) p->fire_valid = 0;
        return CSS_OK;
    }
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
    if (face || bary || vel) p->fire_valid = 0;
    return CSS_OK;
}

int css_particles_set_step(css_parts* p, int64_t step) {
    if (!p || step < 0) return CSS_ERR_INVALID_ARG;
    css_ctx* c = p->ctx;
    p->step = step;
    TRY(c, "set_step", cudaMemcpyAsync(p->dstep, &p->step, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    TRY(c, "set_step", cudaStreamSynchronize(c->stream));
    return CSS_OK;
}

int css_particles_free(css_parts* p) {
    if (!p) return CSS_ERR_INVALID_ARG;
    if (p->graph) cudaGraphExecDestroy(p->graph);
    cudaFree(p->state); cudaFree(p->snap);
    cudaFree(p->fcnt); cudaFree(p->fstart); cudaFree(p->fitems); cudaFree(p->ftmp); cudaFree(p->scan_tmp); cudaFree(p->order);
    cudaFree(p->pcnt); cudaFree(p->pj); cudaFree(p->pd); cudaFree(p->pt); cudaFree(p->dstep); cudaFree(p->dfire);
    delete p;
    return CSS_OK;
}


int css_geodesic_neighbors(css_parts* p, double r_c, int precision, int64_t capacity, int64_t* n_pairs,
                           int64_t* row_start, int32_t* nbr_j, double* dist, double* tangent) {
    Range range_("css_geodesic_neighbors");
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
    Range range_("css_compute_forces");
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
    cudaError_t e = cudaMemcpyAsync(p->snap, p->state, p->state_bytes(), cudaMemcpyDeviceToDevice, p->ctx->stream);
    if (e != cudaSuccess || !p->fire_valid) return e;
    return cudaMemcpyAsync(p->dfire + 8, p->dfire, 8 * sizeof(double), cudaMemcpyDeviceToDevice, p->ctx->stream);
}

cudaError_t snap_restore(css_parts* p) {
    cudaStream_t st = p->ctx->stream;
    cudaError_t e = cudaMemcpyAsync(p->state, p->snap, p->state_bytes(), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && p->fire_valid)
        e = cudaMemcpyAsync(p->dfire, p->dfire + 8, 8 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(p->dstep, &p->step, sizeof(int64_t), cudaMemcpyHostToDevice, st);
}

// per-set integrator kernels of one step: NVE half = 0 before the forces (kick + drift),
// half = 1 after them (kick); overdamped dynamics move after the forces
int enqueue_move(css_parts* p, const css_integrator* it, const double* noise, int half) {
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    const int32_t n = (int32_t)p->n;
    if (it->kind == CSS_INT_FIRE) {
        TRY(c, "fire", cssi::launch_fire_move(p->mesh->view(), n, p->face, p->bary, p->vel, p->force, p->dfire, *it,
                                              half, c->dscal + 1, st));
    } else if (it->kind == CSS_INT_NVE) {
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
                 const double* noise, const GeoPlan& P) {
    css_ctx* c = p->ctx;
    int r = enqueue_move(p, it, noise, 0);
    if (r) return r;
    TRY(c, "reset", cudaMemsetAsync(c->depot, 0, sizeof(double), c->stream));
    r = enqueue_geo(p, rc, prec, 0, 1, pot, P);
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
    Range range_("css_integrate_step");
    if (!p || !pot || !it || bad_prec(precision) || bad_rc(r_c) || n_steps < 0 || it->kind < 0 || it->kind > 4 ||
        !(it->dt > 0.0) || !(it->mass > 0.0) || !(it->lambda > 0.0) || !(it->max_disp > 0.0))
        return CSS_ERR_INVALID_ARG;
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    if (n_steps == 0) return CSS_OK;
    // NVE and FIRE need the force at the current positions
    if ((it->kind == CSS_INT_NVE || it->kind == CSS_INT_FIRE) &&
        !(p->force_valid && p->force_rc == r_c && p->force_prec == precision &&
          memcmp(&p->force_pot, pot, sizeof(css_potential)) == 0)) {
        int rc = css_compute_forces(p, pot, r_c, precision, nullptr, nullptr);
        if (rc) return rc;
    }
    // FIRE starts from (dt, alpha 0.1, no step counted) for new parameters or a new state
    if (it->kind == CSS_INT_FIRE && !(p->fire_valid && memcmp(&p->fire_it, it, sizeof(css_integrator)) == 0)) {
        const double init[8] = {it->dt, 0.1, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        TRY(c, "fire state", cudaMemcpyAsync(p->dfire, init, sizeof(init), cudaMemcpyHostToDevice, st));
        TRY(c, "fire state", cudaStreamSynchronize(st));
        p->fire_valid = 1;
        p->fire_it = *it;
    }
    // host noise is staged in a device buffer that this guard frees on every return path
    struct NoiseBuf {
        double* owned = nullptr;
        ~NoiseBuf() { cudaFree(owned); }
    } staged;
    double* dnoise = nullptr;
    if (noise) {
        const size_t cnt = (size_t)n_steps * p->n * 2;
        if (is_device_ptr(noise)) dnoise = const_cast<double*>(noise);
        else {
            TRY(c, "noise", cudaMalloc(&staged.owned, cnt * sizeof(double)));
            dnoise = staged.owned;
            TRY(c, "noise", cudaMemcpyAsync(dnoise, noise, cnt * sizeof(double), cudaMemcpyHostToDevice, st));
        }
    }
    int retries = 0;
    c->last_counters[5] = 0;
    int rc = CSS_OK;
    for (;;) {
        TRY(c, "snapshot", snap_take(p));
        GeoPlan P;
        rc = ensure_plan(c, precision, p->n, &P);
        if (rc) break;
        TRY(c, "reset", cudaMemsetAsync(c->dscal + 1, 0, sizeof(int), st));
        TRY(c, "reset", cudaMemsetAsync(c->dcount, 0, 8 * sizeof(unsigned long long), st));
        if (!dnoise) {
            // one captured step, kept with the parameters it was captured for, replayed
            std::string key((const char*)pot, sizeof(*pot));
            key.append((const char*)it, sizeof(*it));
            key.append((const char*)&r_c, sizeof(r_c));
            key.append((const char*)&precision, sizeof(precision));
            key.append(plan_key(c, P));
            if (!p->graph || p->graph_key != key) {
                if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
                rc = capture(c, [&]() { return enqueue_step(p, pot, it, r_c, precision, nullptr, P); }, &p->graph);
                if (rc == CSS_OK) p->graph_key = key;
            }
            for (int64_t s = 0; s < n_steps && rc == CSS_OK; ++s) {
                cudaError_t e = cudaGraphLaunch(p->graph, st);
                if (e != cudaSuccess) rc = cuda_fail(c, "graph launch", e);
            }
        } else {
            for (int64_t s = 0; s < n_steps && rc == CSS_OK; ++s)
                rc = enqueue_step(p, pot, it, r_c, precision, dnoise ? dnoise + (size_t)s * p->n * 2 : nullptr, P);
        }
        if (rc) break;
        int status = 0;
        rc = read_status(c, &status);
        if (rc) break;
        if (status == 0) { adapt_default(c); break; }
        if (!grow_for(c, status, &retries)) { rc = status_error(c, status); break; }
        TRY(c, "restore", snap_restore(p));
    }
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
    // the sets as the batched move / bucket kernels see them, and their particle offsets
    cssi::SetView* dviews = nullptr;
    int32_t* doffs = nullptr;
    // captured single step and the parameters it was captured for
    cudaGraphExec_t graph = nullptr;
    std::string graph_key;
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
    std::vector<cssi::SetView> hv;
    std::vector<int32_t> hoff(1, 0);
    for (css_parts* p : b->sets) {
        cssi::SetView v{};
        v.m = p->mesh->view();
        v.face = p->face; v.bary = p->bary; v.vel = p->vel; v.orient = p->orient; v.force = p->force;
        v.fcnt = p->fcnt; v.fstart = p->fstart; v.fitems = p->fitems; v.ftmp = p->ftmp; v.dstep = p->dstep; v.seed = p->seed;
        hv.push_back(v);
        hoff.push_back(hoff.back() + (int32_t)p->n);
    }
    cudaError_t e = cudaMalloc(&b->djobs, n_sets * sizeof(GeoJob));
    if (e == cudaSuccess) e = stage_in(hv.data(), hv.size(), &b->dviews, c->stream);
    if (e == cudaSuccess) e = stage_in(hoff.data(), hoff.size(), &b->doffs, c->stream);
    if (e == cudaSuccess) e = stage_in(hj.data(), hj.size(), &b->job_of_item, c->stream);
    if (e == cudaSuccess) e = stage_in(hs.data(), hs.size(), &b->src_of_item, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { css_batch_free(b); return cuda_fail(c, "batch_create", e); }
    *out = b;
    return CSS_OK;
}

int css_batch_free(css_batch* b) {
    if (!b) return CSS_ERR_INVALID_ARG;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->dviews);
    cudaFree(b->doffs);
    cudaFree(b->djobs);
    cudaFree(b->job_of_item);
    cudaFree(b->src_of_item);
    delete b;
    return CSS_OK;
}

namespace {

int batch_enqueue_forces(css_batch* b, const css_potential* pot, double rc, int prec, const GeoPlan& P) {
    css_ctx* c = b->ctx;
    cudaStream_t st = c->stream;
    TRY(c, "bucket", cssi::launch_batch_bucket(b->dviews, b->doffs, (int)b->sets.size(), b->nitems, st));
    TRY(c, "reset", cudaMemsetAsync(c->depot, 0, sizeof(double), st));
    GeoJob j0 = make_job(b->sets[0], rc, 0, 1, pot);
    return enqueue_passes(c, j0, b->djobs, b->job_of_item, b->src_of_item, b->nitems, prec, P);
}

}  // namespace

int css_batch_step(css_batch* b, const css_potential* pot, const css_integrator* it, double r_c, int precision,
                   int64_t n_steps) {
    Range range_("css_batch_step");
    if (!b || !pot || !it || bad_prec(precision) || bad_rc(r_c) || n_steps < 0 || it->kind < 0 || it->kind > 3 ||
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
    c->last_counters[5] = 0;
    for (;;) {
        for (css_parts* p : b->sets) TRY(c, "snapshot", snap_take(p));
        GeoPlan P;
        int rc = ensure_plan(c, precision, b->nitems, &P);
        if (rc) return rc;
        TRY(c, "reset", cudaMemsetAsync(c->dscal + 1, 0, sizeof(int), st));
        TRY(c, "reset", cudaMemsetAsync(c->dcount, 0, 8 * sizeof(unsigned long long), st));
        if (nve) {   // forces at the starting positions
            rc = batch_enqueue_forces(b, pot, r_c, precision, P);
            if (rc) return rc;
        }
        // one step: every set moves in one launch, buckets in three, forces in the two passes
        const int ns = (int)b->sets.size();
        auto one_step = [&]() -> int {
            TRY(c, "move", cssi::launch_batch_move(b->dviews, b->doffs, ns, b->nitems, *it, 0, c->dscal + 1, st));
            int r = batch_enqueue_forces(b, pot, r_c, precision, P);
            if (r) return r;
            TRY(c, "move", cssi::launch_batch_move(b->dviews, b->doffs, ns, b->nitems, *it, 1, c->dscal + 1, st));
            return CSS_OK;
        };
        std::string key((const char*)pot, sizeof(*pot));
        key.append((const char*)it, sizeof(*it));
        key.append((const char*)&r_c, sizeof(r_c));
        key.append((const char*)&precision, sizeof(precision));
        key.append(plan_key(c, P));
        if (!b->graph || b->graph_key != key) {
            if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
            rc = capture(c, one_step, &b->graph);
            if (rc) return rc;
            b->graph_key = key;
        }
        for (int64_t s = 0; s < n_steps && rc == CSS_OK; ++s) {
            cudaError_t e = cudaGraphLaunch(b->graph, st);
            if (e != cudaSuccess) rc = cuda_fail(c, "graph launch", e);
        }
        if (rc) return rc;
        int status = 0;
        rc = read_status(c, &status);
        if (rc) return rc;
        if (status == 0) { adapt_default(c); break; }
        if (!grow_for(c, status, &retries)) return status_error(c, status);
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


// ------------------------------------------------------------------------------ autotuner
namespace {

// one timed force evaluation of the tuning queue under the context's current shape;
// second-pass overflows grow its pool and repeat
int tune_run(css_ctx* c, const GeoJob* djobs, const GeoJob& j0, const int32_t* job_of_item, const int32_t* src_of_item,
             int32_t nitems, int prec, double* ms) {
    int retries = 0;
    for (;;) {
        GeoPlan P;
        int rc = ensure_plan(c, prec, nitems, &P);
        if (rc) return rc;
        TRY(c, "reset", cudaMemsetAsync(c->dscal + 1, 0, sizeof(int), c->stream));
        TRY(c, "reset", cudaMemsetAsync(c->dcount, 0, 8 * sizeof(unsigned long long), c->stream));
        TRY(c, "reset", cudaMemsetAsync(c->depot, 0, sizeof(double), c->stream));
        rc = enqueue_passes(c, j0, djobs, job_of_item, src_of_item, nitems, prec, P);
        if (rc) return rc;
        int status = 0;
        rc = read_status(c, &status);
        if (rc) return rc;
        if (status == 0) {
            float f = 0.f;
            TRY(c, "tune timing", cudaEventElapsedTime(&f, c->ev_geo0, c->ev_geo1));
            *ms = (double)f;
            return CSS_OK;
        }
        if (!grow_for(c, status, &retries)) return status_error(c, status);
    }
}

}  // namespace

int css_autotune(css_ctx* c, css_parts* const* sets, int32_t n_sets, const css_potential* pot, double r_c,
                 int precision, int32_t reps, int64_t sample, css_launch* best, double* best_ms) {
    Range range_("css_autotune");
    if (!c || !sets || n_sets < 1 || !pot || bad_prec(precision) || bad_rc(r_c) || reps < 1 || sample < 0)
        return CSS_ERR_INVALID_ARG;
    int64_t total = 0;
    for (int k = 0; k < n_sets; ++k) {
        if (!sets[k] || sets[k]->ctx != c) return CSS_ERR_INVALID_ARG;
        total += sets[k]->n;
    }
    if (total < 1 || total > INT32_MAX) return CSS_ERR_INVALID_ARG;
    cudaStream_t st = c->stream;
    // the tuning queue: every source, or about `sample` of them spread evenly over the sets
    const int64_t stride = (sample > 0 && sample < total) ? total / sample : 1;
    std::vector<int32_t> hj, hs;
    std::vector<GeoJob> jobs;
    int64_t g = 0;
    for (int k = 0; k < n_sets; ++k) {
        jobs.push_back(make_job(sets[k], r_c, 0, 1, pot));
        for (int64_t i = 0; i < sets[k]->n; ++i, ++g)
            if (g % stride == 0) { hj.push_back(k); hs.push_back((int32_t)i); }
    }
    GeoJob* djobs = nullptr;
    int32_t *dj = nullptr, *ds = nullptr;
    auto cleanup = [&]() { cudaFree(djobs); cudaFree(dj); cudaFree(ds); };
    cudaError_t e = cudaMalloc(&djobs, jobs.size() * sizeof(GeoJob));
    if (e == cudaSuccess) e = cudaMemcpyAsync(djobs, jobs.data(), jobs.size() * sizeof(GeoJob), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = stage_in(hj.data(), hj.size(), &dj, st);
    if (e == cudaSuccess) e = stage_in(hs.data(), hs.size(), &ds, st);
    for (int k = 0; k < n_sets && e == cudaSuccess; ++k) {
        css_parts* p = sets[k];
        e = cssi::launch_bucket((int32_t)p->n, (int32_t)p->mesh->nf, p->face, p->mesh->frank, p->fcnt, p->fstart, p->fitems, p->ftmp,
                                p->scan_tmp, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(c, "autotune", e); }
    const int32_t nitems = (int32_t)hj.size();
    const cssi::LaunchCfg base = c->cfg;
    constexpr int POOL_UNIT = 2048;   // first-pass windows per warp at table scale 1
    constexpr int TAB_UNIT = 4096;    // global-table slots tried besides tables tied to the pool
    cssi::LaunchCfg pick = base;
    double pick_ms = INFINITY;
    auto measure = [&](const cssi::LaunchCfg& L, double* out) -> int {
        c->cfg = L;
        c->cfg.win_cap2 = std::max(c->cfg.win_cap2, pick.win_cap2);
        double t = 0.0;
        int rc = tune_run(c, djobs, jobs[0], dj, ds, nitems, precision, &t);   // untimed: layout, warm caches
        double m = INFINITY, tot = 0.0;
        // at least `reps` runs, and short launches repeated until ~5 ms were timed (noise)
        for (int r = 0; rc == CSS_OK && (r < reps || (tot < 5.0 && r < 64)); ++r) {
            rc = tune_run(c, djobs, jobs[0], dj, ds, nitems, precision, &t);
            m = std::min(m, t);
            tot += t;
        }
        *out = m;
        return rc;
    };
    int rc = CSS_OK;
    for (int s : {1, 2, 4, 0}) {
        for (int wpc : {2, 4, 8}) {
            const int bps = cssi::geodesic_blocks_per_sm(precision, wpc, s, 1);
            if (bps < 1) continue;
            for (int cps : {0, 1}) {
                if (cps == 1 && bps == 1) continue;   // same shape as "as many as fit"
                cssi::LaunchCfg L = base;
                L.team = 0;
                L.occupancy = 1;
                L.shared_scale = s;
                L.win_cap = POOL_UNIT * (s ? s : 4);   // the pool grows with the patch the tables hold
                L.tab_cap = 0;
                L.warps_per_cta = wpc;
                L.ctas_per_sm = cps;
                L.tile = 1;
                double t = 0.0;
                rc = measure(L, &t);
                if (rc) break;
                if (t < pick_ms) { pick_ms = t; pick = c->cfg; }
                if (s == 0) {   // global tables sized for a patch of about TAB_UNIT / 2 faces
                    cssi::LaunchCfg Lt = L;
                    Lt.tab_cap = TAB_UNIT;
                    rc = measure(Lt, &t);
                    if (rc) break;
                    if (t < pick_ms) { pick_ms = t; pick = c->cfg; }
                }
                // sources deferred for want of pool run twice: try a pool four times larger
                if (c->last_counters[4] * 100 > nitems && L.win_cap * 4 <= (1 << 20)) {
                    L.win_cap *= 4;
                    rc = measure(L, &t);
                    if (rc) break;
                    if (t < pick_ms) { pick_ms = t; pick = c->cfg; }
                }
            }
            if (rc) break;
        }
        if (rc) break;
    }
    // the register-light variant (twice the resident warps, some spills): with global tables
    // (shared tables leave no room for 16 warps per SM) and with the best pick's tables
    for (int variant = 0; variant < 3 && rc == CSS_OK; ++variant) {
        cssi::LaunchCfg T = pick;
        if (variant < 2) {
            T.shared_scale = 0;
            T.win_cap = POOL_UNIT * 4 * (variant == 1 ? 4 : 1);
            if (variant == 1 && T.win_cap <= pick.win_cap && pick.shared_scale == 0) continue;
        } else if (pick.shared_scale == 0) continue;
        for (int wpc : {4, 8}) {
            for (int tab : {0, TAB_UNIT}) {
                if (tab && T.shared_scale) continue;
                cssi::LaunchCfg L = T;
                L.occupancy = 2;
                L.warps_per_cta = wpc;
                L.ctas_per_sm = 0;
                L.tile = 1;
                L.tab_cap = T.shared_scale ? 0 : tab;
                if (cssi::geodesic_blocks_per_sm(precision, wpc, L.shared_scale, 2) < 1) continue;
                double t = 0.0;
                rc = measure(L, &t);
                if (rc) break;
                if (t < pick_ms) { pick_ms = t; pick = c->cfg; }
            }
            if (rc) break;
        }
    }
    // the team form (all warps of a CTA on one source) where the sampled sources are too few to
    // fill the resident warps one warp each
    if (rc == CSS_OK && (int64_t)nitems < 4 * (int64_t)c->sm_count * 8) {
        for (int s : {1, 4, 0}) {
            for (int wpc : {2, 4, 8}) {
                for (int occ : {1, 2}) {
                    if (cssi::geodesic_team_blocks_per_sm(precision, wpc, s, occ) < 1) continue;
                    cssi::LaunchCfg L = base;
                    L.team = 1;
                    L.occupancy = occ;
                    L.shared_scale = s;
                    L.win_cap = POOL_UNIT * (s ? s : 4);
                    L.tab_cap = 0;
                    L.warps_per_cta = wpc;
                    L.ctas_per_sm = 0;
                    L.tile = 1;
                    double t = 0.0;
                    rc = measure(L, &t);
                    if (rc) break;
                    if (t < pick_ms) { pick_ms = t; pick = c->cfg; }
                    // a team's wider waves unfold more windows: sources deferred for want of
                    // pool run twice, so try pools four and sixteen times larger
                    for (int grow = 0; grow < 2 && c->last_counters[4] * 100 > nitems && L.win_cap * 4 <= (1 << 20);
                         ++grow) {
                        L.win_cap *= 4;
                        rc = measure(L, &t);
                        if (rc) break;
                        if (t < pick_ms) { pick_ms = t; pick = c->cfg; }
                    }
                    if (rc) break;
                }
                if (rc) break;
            }
            if (rc) break;
        }
    }
    for (int tile : {2, 4, 8}) {
        if (rc || pick.team) break;   // a team claims one source at a time
        cssi::LaunchCfg L = pick;
        L.tile = tile;
        double t = 0.0;
        rc = measure(L, &t);
        if (rc == CSS_OK && t < pick_ms) { pick_ms = t; pick = c->cfg; }
    }
    cleanup();
    c->cfg = rc == CSS_OK ? pick : base;
    if (rc == CSS_OK) c->cfg_explicit = 1;
    for (int k = 0; k < n_sets; ++k) sets[k]->force_valid = 0;   // forces of the sample only
    if (rc) return rc;
    if (best) css_get_launch(c, best);
    if (best_ms) *best_ms = pick_ms;
    return CSS_OK;
}

// ------------------------------------------------------------------------------ path polylines
int css_trace_geodesics(css_parts* p, int64_t n_paths, const int32_t* src, const double* tangent,
                        const double* length, int32_t max_points, double* points, int32_t* n_points,
                        int32_t* end_face, double* end_bary) {
    Range range_("css_trace_geodesics");
    if (!p || n_paths < 0 || max_points < 2 || (n_paths > 0 && (!src || !tangent || !length || !points || !n_points ||
                                                                 !end_face || !end_bary)))
        return CSS_ERR_INVALID_ARG;
    if (n_paths == 0) return CSS_OK;
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    // the source indices are checked on the host before any kernel reads through them
    std::vector<int32_t> hs((size_t)n_paths);
    std::vector<double> hl((size_t)n_paths), ht(3 * (size_t)n_paths);
    TRY(c, "trace", cudaMemcpy(hs.data(), src, hs.size() * sizeof(int32_t), cudaMemcpyDefault));
    TRY(c, "trace", cudaMemcpy(hl.data(), length, hl.size() * sizeof(double), cudaMemcpyDefault));
    TRY(c, "trace", cudaMemcpy(ht.data(), tangent, ht.size() * sizeof(double), cudaMemcpyDefault));
    for (int64_t k = 0; k < n_paths; ++k) {
        if (hs[k] < 0 || hs[k] >= p->n || !std::isfinite(hl[k]) || hl[k] < 0.0 || !std::isfinite(ht[3 * k]) ||
            !std::isfinite(ht[3 * k + 1]) || !std::isfinite(ht[3 * k + 2])) {
            c->err = "trace_geodesics: path " + std::to_string(k) + " has a bad source index, length or tangent";
            return CSS_ERR_INVALID_ARG;
        }
    }
    int32_t *ds = nullptr, *dn = nullptr, *df = nullptr;
    double *dt = nullptr, *dl = nullptr, *dp = nullptr, *db = nullptr;
    auto cleanup = [&]() { cudaFree(ds); cudaFree(dn); cudaFree(df); cudaFree(dt); cudaFree(dl); cudaFree(dp); cudaFree(db); };
    const size_t np = (size_t)n_paths, npts = np * (size_t)max_points;
    cudaError_t e = stage_in(hs.data(), np, &ds, st);
    if (e == cudaSuccess) e = stage_in(hl.data(), np, &dl, st);
    if (e == cudaSuccess) e = stage_in(ht.data(), 3 * np, &dt, st);
    if (e == cudaSuccess) e = cudaMalloc(&dp, 3 * npts * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dn, np * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&df, np * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&db, 3 * np * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(dp, 0, 3 * npts * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dscal + 1, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = cssi::launch_trace(p->mesh->view(), n_paths, p->face, p->bary, ds, dt, dl, max_points, dp, dn, df, db,
                               c->dscal + 1, st);
    if (e == cudaSuccess) e = copy_out(points, dp, 3 * npts, st);
    if (e == cudaSuccess) e = copy_out(n_points, dn, np, st);
    if (e == cudaSuccess) e = copy_out(end_face, df, np, st);
    if (e == cudaSuccess) e = copy_out(end_bary, db, 3 * np, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->hstat, c->dscal + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(c, "trace_geodesics", e);
    if (*c->hstat) return status_error(c, *c->hstat);
    return CSS_OK;
}

// ------------------------------------------------------------------ shortest-path polylines
namespace {

constexpr int PATH_MAX_LEGS = 32;

// device scratch of one path extraction, freed on every exit
struct PathBufs {
    std::vector<void*> ptrs;
    template <class T>
    cudaError_t alloc(T** p, size_t n) {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~PathBufs() { for (void* q : ptrs) cudaFree(q); }
};

// One launch of the path instantiation of the neighbour kernel over the distinct sources
// (us, on the device as dus): rows in the set's pair slab, legs per (rank in us, row slot).
int run_path_kernel(css_parts* p, double rc, const std::vector<int32_t>& us, const int32_t* dus, int win_cap,
                    int32_t* dlnum, int32_t* dlfk, double* dldir, double* dllen, int* status) {
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    const int nus = (int)us.size();
    int le, lv, lf, fcap, emcap;
    const size_t stride = cssi::geo_ws_bytes_per_warp(CSS_FP64, win_cap, 0, &le, &lv, &lf, &fcap, &emcap);
    const size_t lstride = cssi::geo_link_bytes_per_warp(lv);
    const int wpc = 8;
    const int nwarps = std::min(c->sm_count * wpc, ((nus + wpc - 1) / wpc) * wpc);
    PathBufs B;
    char *base = nullptr, *lbase = nullptr;
    uint32_t* gen = nullptr;
    TRY(c, "paths workspace", B.alloc(&base, (size_t)nwarps * stride));
    TRY(c, "paths workspace", B.alloc(&lbase, (size_t)nwarps * lstride));
    TRY(c, "paths workspace", B.alloc(&gen, (size_t)nwarps));
    TRY(c, "paths workspace", cudaMemsetAsync(base, 0, (size_t)nwarps * stride, st));
    TRY(c, "paths workspace", cudaMemsetAsync(gen, 0, (size_t)nwarps * sizeof(uint32_t), st));
    cssi::GeoWs g{};
    g.shared = 0;
    g.base = base;
    g.stride = stride;
    g.log_eh = le; g.log_vh = lv; g.log_fh = lf;
    g.wcap = win_cap; g.fcap = fcap; g.emcap = emcap;
    g.gen = gen;
    g.nwarps = nwarps;
    g.occupancy = 1;
    g.lbase = lbase;
    g.lstride = lstride;
    TRY(c, "bucket", cssi::launch_bucket((int32_t)p->n, (int32_t)p->mesh->nf, p->face, p->mesh->frank, p->fcnt,
                                         p->fstart, p->fitems, p->ftmp, p->scan_tmp, st));
    GeoJob j = make_job(p, rc, 1, 0, nullptr);
    j.order = dus;
    j.lmax = PATH_MAX_LEGS;
    j.lnum = dlnum; j.lfk = dlfk; j.ldir = dldir; j.llen = dllen;
    cssi::GeoQueue q{nullptr, nullptr, nus, nullptr, nullptr, nullptr, nullptr, 1};
    TRY(c, "reset", cudaMemsetAsync(c->dscal, 0, 2 * sizeof(int), st));
    TRY(c, "reset", cudaMemsetAsync(c->dcount, 0, 8 * sizeof(unsigned long long), st));
    TRY(c, "paths", cssi::launch_geodesic_links(j, q, g, wpc, nwarps / wpc, c->dscal, c->dscal + 1, c->dcount, st));
    return read_status(c, status);
}

}  // namespace

int css_geodesic_paths(css_parts* p, double r_c, int64_t n_pairs, const int32_t* src, const int32_t* dst,
                       int32_t max_points, double* points, int32_t* n_points, int32_t* n_legs, double* dist,
                       double* gap) {
    Range range_("css_geodesic_paths");
    if (!p || bad_rc(r_c) || n_pairs < 0 || max_points < 2 ||
        (n_pairs > 0 && (!src || !dst || !points || !n_points || !n_legs || !dist || !gap)))
        return CSS_ERR_INVALID_ARG;
    if (n_pairs == 0) return CSS_OK;
    css_ctx* c = p->ctx;
    cudaStream_t st = c->stream;
    const size_t np = (size_t)n_pairs;
    std::vector<int32_t> hs(np), hd(np);
    TRY(c, "paths", cudaMemcpy(hs.data(), src, np * sizeof(int32_t), cudaMemcpyDefault));
    TRY(c, "paths", cudaMemcpy(hd.data(), dst, np * sizeof(int32_t), cudaMemcpyDefault));
    for (size_t k = 0; k < np; ++k)
        if (hs[k] < 0 || hs[k] >= p->n || hd[k] < 0 || hd[k] >= p->n || hs[k] == hd[k]) {
            c->err = "geodesic_paths: pair " + std::to_string(k) + " has a bad or repeated particle index";
            return CSS_ERR_INVALID_ARG;
        }
    std::vector<int32_t> us(hs);
    std::sort(us.begin(), us.end());
    us.erase(std::unique(us.begin(), us.end()), us.end());
    const int nus = (int)us.size();
    PathBufs B;
    int32_t* dus = nullptr;
    TRY(c, "paths", B.alloc(&dus, us.size()));
    TRY(c, "paths", cudaMemcpyAsync(dus, us.data(), us.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    // the kernel, grown until neither the window pool nor the pair rows overflow
    int win_cap = next_pow2(std::max(c->cfg.win_cap2, 16384));
    int32_t *dlnum = nullptr, *dlfk = nullptr;
    double *dldir = nullptr, *dllen = nullptr;
    int cap = 0;
    for (int attempt = 0;; ++attempt) {
        int rc = ensure_pairs(p, c->pair_cap);
        if (rc) return rc;
        cap = p->pair_cap_alloc;
        PathBufs L;
        const size_t slots = (size_t)nus * cap;
        TRY(c, "paths", L.alloc(&dlnum, slots));
        TRY(c, "paths", L.alloc(&dlfk, slots * PATH_MAX_LEGS));
        TRY(c, "paths", L.alloc(&dldir, 2 * slots * PATH_MAX_LEGS));
        TRY(c, "paths", L.alloc(&dllen, slots * PATH_MAX_LEGS));
        int status = 0;
        rc = run_path_kernel(p, r_c, us, dus, win_cap, dlnum, dlfk, dldir, dllen, &status);
        if (rc) return rc;
        if (status == 0) {
            // keep the leg buffers: hand them to the outer scope
            B.ptrs.insert(B.ptrs.end(), L.ptrs.begin(), L.ptrs.end());
            L.ptrs.clear();
            break;
        }
        if (attempt >= MAX_RETRY) return status_error(c, status);
        if (status & (css::ST_WIN_OVERFLOW | css::ST_HASH_OVERFLOW | css::ST_ITER_LIMIT)) {
            if (win_cap >= WIN_CAP_MAX) return status_error(c, status);
            win_cap *= 2;
        } else if (status & css::ST_PAIR_OVERFLOW) {
            c->pair_cap *= 2;
        } else {
            return status_error(c, status);
        }
    }
    // rows and legs of the distinct sources
    const size_t slots = (size_t)nus * cap;
    std::vector<int32_t> pcnt(p->n), pj((size_t)p->n * cap), lnum(slots), lfk(slots * PATH_MAX_LEGS);
    std::vector<double> pd((size_t)p->n * cap), ldir(2 * slots * PATH_MAX_LEGS), llen(slots * PATH_MAX_LEGS);
    TRY(c, "paths", cudaMemcpyAsync(pcnt.data(), p->pcnt, pcnt.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRY(c, "paths", cudaMemcpyAsync(pj.data(), p->pj, pj.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRY(c, "paths", cudaMemcpyAsync(pd.data(), p->pd, pd.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TRY(c, "paths", cudaMemcpyAsync(lnum.data(), dlnum, lnum.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRY(c, "paths", cudaMemcpyAsync(lfk.data(), dlfk, lfk.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRY(c, "paths", cudaMemcpyAsync(ldir.data(), dldir, ldir.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TRY(c, "paths", cudaMemcpyAsync(llen.data(), dllen, llen.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TRY(c, "paths", cudaStreamSynchronize(st));
    // the legs of every requested pair, from the target back to the source
    std::vector<int64_t> first(np + 1, 0);
    std::vector<int32_t> s_fk, s_pi, n_fk, n_pi;
    std::vector<double> l_dir, l_len;
    std::vector<double> hdist(np, INFINITY);
    for (size_t k = 0; k < np; ++k) {
        first[k] = (int64_t)s_fk.size();
        const int i = hs[k], jj = hd[k];
        const int r = (int)(std::lower_bound(us.begin(), us.end(), i) - us.begin());
        const int cnt = std::min(pcnt[i], cap);
        int pos = -1;
        for (int a = 0; a < cnt; ++a)
            if (pj[(size_t)i * cap + a] == jj) { pos = a; break; }
        if (pos < 0) continue;   // not within the cutoff
        hdist[k] = pd[(size_t)i * cap + pos];
        const size_t o = (size_t)r * cap + pos;
        const int nl = lnum[o];
        if (nl <= 0) {
            c->err = "geodesic_paths: the path of pair " + std::to_string(k) +
                     (nl == -1 ? " has more legs than the limit" : " lost a vertex link");
            return CSS_ERR_ITER_LIMIT;
        }
        for (int l = 0; l < nl; ++l) {
            const size_t a = o * PATH_MAX_LEGS + l;
            s_fk.push_back(lfk[a]);
            s_pi.push_back(l == 0 ? jj : -1);
            l_dir.push_back(ldir[2 * a]);
            l_dir.push_back(ldir[2 * a + 1]);
            l_len.push_back(llen[a]);
            if (l + 1 < nl) { n_fk.push_back(lfk[a + 1]); n_pi.push_back(-1); }
            else { n_fk.push_back(-1); n_pi.push_back(i); }
        }
    }
    first[np] = (int64_t)s_fk.size();
    const int64_t nleg = first[np];
    std::vector<int32_t> nrec(nleg);
    std::vector<double> rec((size_t)nleg * max_points * 3), sw(3 * (size_t)nleg), nw(3 * (size_t)nleg), lg(nleg);
    if (nleg > 0) {
        int32_t *d_sfk, *d_spi, *d_nfk, *d_npi, *d_nrec;
        double *d_dir, *d_len, *d_rec, *d_sw, *d_nw, *d_gap;
        TRY(c, "paths", B.alloc(&d_sfk, nleg));
        TRY(c, "paths", B.alloc(&d_spi, nleg));
        TRY(c, "paths", B.alloc(&d_nfk, nleg));
        TRY(c, "paths", B.alloc(&d_npi, nleg));
        TRY(c, "paths", B.alloc(&d_nrec, nleg));
        TRY(c, "paths", B.alloc(&d_dir, 2 * nleg));
        TRY(c, "paths", B.alloc(&d_len, nleg));
        TRY(c, "paths", B.alloc(&d_rec, rec.size()));
        TRY(c, "paths", B.alloc(&d_sw, sw.size()));
        TRY(c, "paths", B.alloc(&d_nw, nw.size()));
        TRY(c, "paths", B.alloc(&d_gap, lg.size()));
        TRY(c, "paths", cudaMemcpyAsync(d_sfk, s_fk.data(), nleg * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        TRY(c, "paths", cudaMemcpyAsync(d_spi, s_pi.data(), nleg * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        TRY(c, "paths", cudaMemcpyAsync(d_nfk, n_fk.data(), nleg * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        TRY(c, "paths", cudaMemcpyAsync(d_npi, n_pi.data(), nleg * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        TRY(c, "paths", cudaMemcpyAsync(d_dir, l_dir.data(), 2 * nleg * sizeof(double), cudaMemcpyHostToDevice, st));
        TRY(c, "paths", cudaMemcpyAsync(d_len, l_len.data(), nleg * sizeof(double), cudaMemcpyHostToDevice, st));
        TRY(c, "paths", cssi::launch_legs(p->mesh->view(), nleg, p->face, p->bary, d_sfk, d_spi, d_dir, d_len, d_nfk,
                                          d_npi, max_points, d_rec, d_nrec, d_sw, d_nw, d_gap, st));
        TRY(c, "paths", cudaMemcpyAsync(nrec.data(), d_nrec, nleg * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TRY(c, "paths", cudaMemcpyAsync(rec.data(), d_rec, rec.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        TRY(c, "paths", cudaMemcpyAsync(sw.data(), d_sw, sw.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        TRY(c, "paths", cudaMemcpyAsync(nw.data(), d_nw, nw.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        TRY(c, "paths", cudaMemcpyAsync(lg.data(), d_gap, lg.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        TRY(c, "paths", cudaStreamSynchronize(st));
    }
    // polylines from the source: its position, then the legs in reverse order, each reversed
    std::vector<double> out(np * (size_t)max_points * 3, 0.0);
    std::vector<int32_t> onp(np, 0), onl(np, 0);
    std::vector<double> ogap(np, 0.0);
    for (size_t k = 0; k < np; ++k) {
        const int64_t a0 = first[k], a1 = first[k + 1];
        if (a1 == a0) continue;
        int64_t n = 0;
        double g = 0.0;
        auto put = [&](const double* w) {
            if (n < max_points) for (int a = 0; a < 3; ++a) out[3 * (k * max_points + n) + a] = w[a];
            ++n;
        };
        put(&nw[3 * (a1 - 1)]);
        for (int64_t l = a1 - 1; l >= a0; --l) {
            if (nrec[l] < 0) {
                c->err = "geodesic_paths: walking a leg of pair " + std::to_string(k) + " failed (" +
                         std::to_string(nrec[l]) + ")";
                return CSS_ERR_ITER_LIMIT;
            }
            for (int r = std::min<int>(nrec[l], max_points) - 1; r >= 0; --r) put(&rec[3 * ((size_t)l * max_points + r)]);
            if (nrec[l] > max_points) n += nrec[l] - max_points;   // counted, not stored
            put(&sw[3 * l]);
            g = std::max(g, lg[l]);
        }
        onp[k] = (int32_t)std::min<int64_t>(n, INT32_MAX);
        onl[k] = (int32_t)(a1 - a0);
        ogap[k] = g;
    }
    TRY(c, "paths", cudaMemcpy(points, out.data(), out.size() * sizeof(double), cudaMemcpyDefault));
    TRY(c, "paths", cudaMemcpy(n_points, onp.data(), np * sizeof(int32_t), cudaMemcpyDefault));
    TRY(c, "paths", cudaMemcpy(n_legs, onl.data(), np * sizeof(int32_t), cudaMemcpyDefault));
    TRY(c, "paths", cudaMemcpy(dist, hdist.data(), np * sizeof(double), cudaMemcpyDefault));
    TRY(c, "paths", cudaMemcpy(gap, ogap.data(), np * sizeof(double), cudaMemcpyDefault));
    return CSS_OK;
}
