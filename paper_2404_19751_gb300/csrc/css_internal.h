// css_internal.h -- host-side objects behind the C ABI handles and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/css.h"
#include "css_dev.cuh"

struct css_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int own_stream = 0;
    int sm_count = 0;
    std::string err;
    // neighbour/force workspace (grown on demand)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    uint32_t* ws_gen = nullptr;      // per warp generation counters
    int ws_warps = 0;
    int64_t ws_key = -1;             // layout the workspace bytes were zeroed for
    int warps_per_cta = 4;
    int win_cap = 2048;              // windows per warp workspace
    int pair_cap = 64;               // pairs per source slab
    int shared_tables = 1;           // try shared-memory tables first
    // small device scalars: [0] work counter, [1] status, [2..] counters
    int* dscal = nullptr;
    unsigned long long* dcount = nullptr;   // 8 counters
    double* depot = nullptr;
    int* hstat = nullptr;                   // pinned mirror of status
    unsigned long long* hcount = nullptr;   // pinned mirror of counters
    int64_t last_counters[6] = {0, 0, 0, 0, 0, 0};
    cudaEvent_t ev_geo0 = nullptr, ev_geo1 = nullptr;   // around the neighbour/force kernel
    int ev_valid = 0;
};

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
    int32_t* scan_tmp = nullptr;
    int32_t* order = nullptr;   // source processing order (n)
    int64_t* dstep = nullptr;   // device copy of the step counter (Philox counter word)
    // pair slab
    int32_t* pcnt = nullptr;    // n
    int32_t* pj = nullptr;
    double* pd = nullptr;
    double* pt = nullptr;
    int pair_cap_alloc = 0;
    int global_tables = 0;      // this set's patches overflowed the shared-memory tables
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
};

struct GeoWs {
    int shared;              // keyed tables in shared memory (else in the global slice)
    char* base;
    size_t stride;           // bytes per warp
    int log_eh, log_vh, log_fh;
    int wcap, fcap, emcap;
    uint32_t* gen;
    int nwarps;
};

// geodesic.cu
size_t geo_ws_bytes_per_warp(int precision, int win_cap, int* log_eh, int* log_vh, int* log_fh,
                             int* fcap, int* emcap);
cudaError_t launch_geodesic(const GeoJob& job0, const GeoJob* djobs, const int32_t* job_of_item,
                            const int32_t* src_of_item, int32_t nitems, int precision,
                            const GeoWs& ws, int warps_per_cta, int nctas, int* work_counter,
                            int* status, unsigned long long* counters, cudaStream_t st);
int geodesic_blocks_per_sm(int precision, int warps_per_cta, int shared);
cudaError_t launch_pairs_compact(int32_t n, const int32_t* pcnt, const int32_t* pj, const double* pd,
                                 const double* pt, int pair_cap, const int64_t* row_start,
                                 int32_t* out_j, double* out_d, double* out_t, cudaStream_t st);

// dynamics.cu
cudaError_t launch_bucket(int32_t n, int32_t nf, const int32_t* face, int32_t* fcnt, int32_t* fstart,
                          int32_t* fitems, int32_t* scan_tmp, cudaStream_t st);
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

// peak.cu
cudaError_t measure_fma_peak(int precision, int sm_count, cudaStream_t st, double* flops);

// mesh_prep.cu
int build_mesh(css_ctx* ctx, const double* dX, int64_t nv, const int32_t* dF, int64_t nf,
               const double* period, css_mesh* m);

}  // namespace cssi
