// css_internal.h -- host-side objects behind the C ABI handles and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/css.h"
#include "css_dev.cuh"

namespace cssi {
// Launch shape of the neighbour / force evaluation.  The first pass runs every source
// with per-warp tables in shared memory (scaled by `shared_scale`, 0: global tables) and a
// window pool of `win_cap`; sources whose patch overflows either are deferred to a
// second pass with global tables and a pool of `win_cap2`, on fewer warps.
struct LaunchCfg {
    int warps_per_cta = 4;   // first pass
    int ctas_per_sm = 0;     // 0: as many as fit
    int tile = 1;            // work items a warp claims at a time
    int shared_scale = 1;    // 0, 1, 2, 4, 8
    int win_cap = 2048;
    int win_cap2 = 16384;
    int warps2_per_sm = 2;   // second pass: warps per SM (one CTA each)
    int occupancy = 1;       // register budget of the first pass: 1 (255 regs) or 2 (128 regs)
    int tab_cap = 0;         // first pass with global tables: table slots (0: tied to win_cap)
    int team = 0;            // 1: the warps of a CTA work on one source together (team form)
};
// a second-pass workspace (global tables)
struct WsBuf {
    void* ws = nullptr;
    size_t bytes = 0;
    uint32_t* gen = nullptr;
    int warps = 0;
    int64_t key = -1;        // layout the bytes were zeroed for
};
}  // namespace cssi

struct css_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int own_stream = 0;
    int sm_count = 0;
    std::string err;
    // neighbour/force workspaces of the two passes (grown on demand)
    cssi::WsBuf ws1, ws2;
    cssi::LaunchCfg cfg;
    std::map<int64_t, int> bps_cache;   // resident CTAs per SM by (precision, shape)
    int cfg_explicit = 0;               // the shape was set or tuned (no automatic adaptation)
    int pair_cap = 64;               // pairs per source slab
    // deferral list of the first pass (one entry per work item at most)
    int32_t* defer = nullptr;
    int64_t defer_cap = 0;
    // small device scalars: [0] first-pass work counter, [1] status, [2] deferred count,
    // [3] second-pass work counter
    int* dscal = nullptr;
    unsigned long long* dcount = nullptr;   // 8 counters
    double* depot = nullptr;
    int* hstat = nullptr;                   // pinned mirror of status
    unsigned long long* hcount = nullptr;   // pinned mirror of counters
    int64_t last_counters[6] = {0, 0, 0, 0, 0, 0};
    cudaEvent_t ev_geo0 = nullptr, ev_geo1 = nullptr;   // around the neighbour/force kernel
    int ev_valid = 0;
    // orders work on another stream after what is queued on `stream` (made at creation so
    // that the allocation-free entry point creates nothing)
    cudaEvent_t ev_order = nullptr;
};

namespace cssi {
struct VhmOp;   // operators of the approximate solver (vhm.cu), built on first use
void vhm_free(css_mesh* m);
}  // namespace cssi

struct css_mesh {
    css_ctx* ctx = nullptr;
    int64_t nv = 0, nf = 0, ne = 0, npseudo = 0;
    int periodic = 0;
    double per[2] = {0, 0};
    // device arrays
    css::HeRec* he = nullptr;
    int32_t* twin = nullptr;
    int32_t* edge = nullptr;
    int32_t* fv = nullptr;
    double* lay = nullptr;
    double* frame = nullptr;
    double* theta = nullptr;
    uint8_t* pseudo = nullptr;
    uint8_t* bnd = nullptr;
    int32_t* ring_start = nullptr;
    int32_t* ring = nullptr;
    double* X = nullptr;
    css::HeRec32* he32 = nullptr;
    float* lay32 = nullptr;
    int32_t* frank = nullptr;   // nf: Morton rank of each face
    float2* cang = nullptr;     // 3 nf: corner (start, width) around its vertex
    cssi::VhmOp* vhm = nullptr;
    css::DMesh view() const;
};

struct css_parts {
    css_ctx* ctx = nullptr;
    css_mesh* mesh = nullptr;
    int64_t n = 0;
    uint64_t seed = 0;
    int64_t step = 0;
    int force_valid = 0;
    double force_rc = 0.0;
    int force_prec = -1;
    css_potential force_pot{};
    // device arrays (bary, vel, orient, force, face live in one block `state`)
    void* state = nullptr;
    void* snap = nullptr;       // copy of `state` taken before a multi-step call
    size_t state_bytes() const { return (size_t)n * (12 * sizeof(double) + sizeof(int32_t)); }
    int32_t* face = nullptr;
    double* bary = nullptr;     // 3 n
    double* vel = nullptr;      // 3 n
    double* orient = nullptr;   // 3 n
    double* force = nullptr;    // 3 n
    int32_t* fcnt = nullptr;    // nf (kept at zero between uses)
    int32_t* fstart = nullptr;  // nf + 1
    int32_t* fitems = nullptr;  // n
    int32_t* ftmp = nullptr;    // n, scratch of the bucket scatter
    int32_t* scan_tmp = nullptr;
    int32_t* order = nullptr;   // source processing order (n)
    int64_t* dstep = nullptr;   // device copy of the step counter (Philox counter word)
    double* dfire = nullptr;    // FIRE state: 8 live doubles, then their snapshot
    int fire_valid = 0;         // the FIRE state belongs to fire_it and the current particles
    css_integrator fire_it{};
    // pair slab
    int32_t* pcnt = nullptr;    // n
    int32_t* pj = nullptr;
    double* pd = nullptr;
    double* pt = nullptr;
    int pair_cap_alloc = 0;
    // captured single-step graph and the launch parameters it was captured for
    cudaGraphExec_t graph = nullptr;
    std::string graph_key;
};

namespace cssi {

// parameters of one neighbour / force launch over one particle set
struct GeoJob {
    css::DMesh m;
    int32_t n;
    const int32_t* face;
    const double* bary;
    const int32_t* fstart;
    const int32_t* fitems;
    const int32_t* order;
    double rc;
    // outputs
    int32_t want_pairs;
    int32_t pair_cap;
    int32_t* pcnt;
    int32_t* pj;
    double* pd;
    double* pt;
    int32_t want_forces;
    css_potential pot;
    double* force;
    double* epot;
    // path launches: for the pair in slot o of the row of the item'th source, its legs
    // (lnum[o], at most lmax) as 4 * face + corner (corner 3: the target point), unit
    // direction and length at lfk/ldir/llen[o * lmax + leg]; lnum -1: more legs than lmax
    int32_t lmax = 0;
    int32_t* lnum = nullptr;
    int32_t* lfk = nullptr;
    double* ldir = nullptr;
    double* llen = nullptr;
};

// one particle set as the batched move / bucket kernels see it
struct SetView {
    css::DMesh m;
    int32_t* face;
    double* bary;
    double* vel;
    double* orient;
    double* force;
    int32_t* fcnt;
    int32_t* fstart;
    int32_t* fitems;
    int32_t* ftmp;
    int64_t* dstep;
    uint64_t seed;
};

// where a launch takes its work items from
struct GeoQueue {
    const int32_t* job_of_item;   // NULL: one job
    const int32_t* src_of_item;   // NULL: item = source index (or the job's order)
    int32_t nitems;
    const int32_t* item_list;     // second pass: items from the deferral list ...
    const int* item_count;        // ... of this many entries (device)
    int32_t* defer_list;          // first pass: where overflowing items go (NULL: report)
    int* defer_count;
    int tile;
};

struct GeoWs {
    int shared;              // scale of the keyed tables in shared memory, 0: global slice
    char* base;
    size_t stride;           // bytes per warp
    int log_eh, log_vh, log_fh;
    int wcap, fcap, emcap;
    uint32_t* gen;
    int nwarps;
    int occupancy;           // kernel variant: 1 (255 registers a thread) or 2 (128)
    char* lbase = nullptr;   // path launches: per-warp vertex link arrays (lstride bytes a warp)
    size_t lstride = 0;
};

// geodesic.cu
size_t geo_ws_bytes_per_warp(int precision, int win_cap, int tab_cap, int* log_eh, int* log_vh, int* log_fh,
                             int* fcap, int* emcap);
cudaError_t launch_geodesic(const GeoJob& job0, const GeoJob* djobs, const GeoQueue& q, int precision,
                            const GeoWs& ws, int warps_per_cta, int nctas, int* work_counter,
                            int* status, unsigned long long* counters, cudaStream_t st);
// the FP64, global-table kernel that also records the legs of every pair's path
size_t geo_link_bytes_per_warp(int log_vh);
cudaError_t launch_geodesic_links(const GeoJob& job, const GeoQueue& q, const GeoWs& ws, int warps_per_cta,
                                  int nctas, int* work_counter, int* status, unsigned long long* counters,
                                  cudaStream_t st);
int geodesic_blocks_per_sm(int precision, int warps_per_cta, int shared_scale, int occupancy);
// team form of the first pass: all warps of a CTA (2..8) on one source; ws counts teams
cudaError_t launch_geodesic_team(const GeoJob& job0, const GeoJob* djobs, const GeoQueue& q, int precision,
                                 const GeoWs& ws, int warps_per_cta, int nctas, int* work_counter, int* status,
                                 unsigned long long* counters, cudaStream_t st);
int geodesic_team_blocks_per_sm(int precision, int warps_per_cta, int shared_scale, int occupancy);
size_t geodesic_team_shared_bytes(int precision, int warps_per_cta, int shared_scale);
size_t geodesic_shared_bytes(int precision, int warps_per_cta, int shared_scale);
cudaError_t launch_pairs_compact(int32_t n, const int32_t* pcnt, const int32_t* pj, const double* pd,
                                 const double* pt, int pair_cap, const int64_t* row_start,
                                 int32_t* out_j, double* out_d, double* out_t, cudaStream_t st);

// dynamics.cu
// particles bucketed by face rank: fstart (nf + 1) is indexed by frank[face] (NULL: by
// face), fitems lists the particles in rank order
// face buckets of n particles: counts, offsets, then the particles of each face in index
// order (ftmp: n ints of scratch for the unordered scatter)
cudaError_t launch_bucket(int32_t n, int32_t nf, const int32_t* face, const int32_t* frank, int32_t* fcnt,
                          int32_t* fstart, int32_t* fitems, int32_t* ftmp, int32_t* scan_tmp, cudaStream_t st);
size_t scan_tmp_ints(int64_t count);
cudaError_t launch_scan_i32(const int32_t* in, int32_t* out_excl, int64_t count, int32_t* tmp,
                            cudaStream_t st);
cudaError_t launch_scan_rows(const int32_t* cnt, int64_t* row_start, int32_t n, cudaStream_t st);
cudaError_t launch_nve_kick_drift(const css::DMesh& m, int32_t n, int32_t* face, double* bary,
                                  double* vel, const double* force, css_integrator it, int* status,
                                  cudaStream_t st);
cudaError_t launch_nve_kick(int32_t n, double* vel, const double* force, css_integrator it,
                            cudaStream_t st);
cudaError_t launch_overdamped_move(const css::DMesh& m, int32_t n, int32_t* face, double* bary,
                                   double* orient, const double* force, css_integrator it,
                                   uint64_t seed, const int64_t* dstep, const double* noise, int* status,
                                   cudaStream_t st);
cudaError_t launch_step_inc(int64_t* dstep, cudaStream_t st);
// FIRE minimiser step halves (half 0: reductions, control, mixing, kick and drift; half 1:
// the second kick); fire_state: 8 doubles on the device (see dynamics.cu)
cudaError_t launch_fire_move(const css::DMesh& m, int32_t n, int32_t* face, double* bary, double* vel,
                             const double* force, double* fire_state, css_integrator it, int half, int* status,
                             cudaStream_t st);
// straightest-walk polylines of npaths paths (see css_trace_geodesics)
// walks the legs of shortest paths (see k_legs in dynamics.cu)
cudaError_t launch_legs(const css::DMesh& m, int64_t nleg, const int32_t* pface, const double* pbary,
                        const int32_t* start_fk, const int32_t* start_pi, const double* dir, const double* len,
                        const int32_t* next_fk, const int32_t* next_pi, int cap, double* rec, int32_t* nrec,
                        double* start_w, double* next_w, double* gap, cudaStream_t st);
cudaError_t launch_trace(const css::DMesh& m, int64_t npaths, const int32_t* pface, const double* pbary,
                         const int32_t* src, const double* tan, const double* len, int cap, double* pts,
                         int32_t* npts, int32_t* end_face, double* end_bary, int* status, cudaStream_t st);
// bitwise change of an uploaded state against the current one (flag |= 1 positions, 2 velocities)
cudaError_t launch_state_diff(int32_t n, const int32_t* nf, const int32_t* of, const double* nb, const double* ob,
                              const double* nv, const double* ov, int* flag, cudaStream_t st);
// batched forms over the sets of a batch: item k belongs to set s with offs[s] <= k < offs[s+1]
// (offs has nsets + 1 entries on the device; total = offs[nsets])
cudaError_t launch_batch_bucket(const SetView* sv, const int32_t* offs, int nsets, int64_t total, cudaStream_t st);
cudaError_t launch_batch_move(const SetView* sv, const int32_t* offs, int nsets, int64_t total, css_integrator it,
                              int half, int* status, cudaStream_t st);

// peak.cu
cudaError_t measure_fma_peak(int precision, int sm_count, cudaStream_t st, double* flops);

// mesh_prep.cu
int build_mesh(css_ctx* ctx, const double* dX, int64_t nv, const int32_t* dF, int64_t nf,
               const double* period, css_mesh* m);

}  // namespace cssi
