/*
 * css.h -- C ABI of the curved-surface geodesic molecular-dynamics library
 * (GB300 / sm_103a CUDA).
 *
 * The library implements the per-timestep hot path of particle simulations on
 * triangulated surfaces (Webb & Sussman, "curvedSpaceSim", arXiv:2404.19751):
 *   - exact polyhedral geodesic distances l_ij and initial tangents from every
 *     particle to every particle within a cutoff, by continuous window
 *     propagation over planar unfoldings of the mesh          (Sec. 2.2, 3.1)
 *   - pair forces  F_i = sum_j -U'(l_ij) grad_{x_i} l_ij      (Sec. 2.1, 3.1)
 *   - the straightest face-walk "shift" with parallel transport, driving
 *     velocity-Verlet NVE, Brownian and active Brownian dynamics (Sec. 2.1, 3.2)
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: CSS_OK (0) or a negative CSS_ERR_*
 *     code; none aborts.  css_last_error() gives a one-line message.
 *   - Pointers are plain host or CUDA device pointers; the library detects which
 *     (cudaPointerGetAttributes).  Inputs are copied into library-owned device
 *     memory; outputs go to caller-owned buffers.  A call that writes to host
 *     memory synchronises the context stream before returning.
 *   - All GPU work is enqueued on the stream given to css_create (NULL: the
 *     library creates and owns a non-blocking stream; the legacy default stream
 *     cannot hold a graph capture).  Objects must not be used from two host
 *     threads at once.
 *   - Positions are (face index, barycentric triple); vectors (velocities,
 *     orientations, forces, tangents) are world-frame 3-vectors lying in the
 *     plane of the particle's current face (Sec. 3.2).
 *   - Faces are vertex-index triples, counter-clockwise seen from the side the
 *     surface normal points to; the mesh must be an oriented 2-manifold,
 *     optionally with boundary (Sec. 2.2 assumes closed surfaces; open edges
 *     reflect the face walk) or periodic in x and y.
 */
#ifndef CSS_H
#define CSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define CSS_OK                    0
#define CSS_ERR_INVALID_ARG      -1   /* bad size, index, NaN, null pointer        */
#define CSS_ERR_NONMANIFOLD      -2   /* edge in >2 faces, flipped face, zero area  */
#define CSS_ERR_OOM              -3   /* device allocation failed                   */
#define CSS_ERR_CUDA             -4   /* a CUDA runtime call failed                 */
#define CSS_ERR_CAPACITY         -5   /* caller buffer too small (see n_pairs)      */
#define CSS_ERR_QUEUE_OVERFLOW   -6   /* window workspace exhausted after retries   */
#define CSS_ERR_ITER_LIMIT       -7   /* a device loop reached its iteration cap    */
#define CSS_ERR_NO_DEVICE        -8   /* no CUDA device / wrong architecture        */

/* ---------------------------------------------------------------- enums */
#define CSS_FP64 0   /* every window, distance and walk operation in FP64            */
#define CSS_FP32 1   /* FP32 window arithmetic; FP64 kept for unfolded source
                        coordinates, near-degenerate predicates and the face walk  */

#define CSS_POT_HARMONIC 0   /* U = eps (1 - l/sigma)^2            for l < r_cut     */
#define CSS_POT_WCA      1   /* U = 4 eps ((s/l)^12 - (s/l)^6) + eps for l < r_cut   */
#define CSS_POT_GAUSSIAN 2   /* U = A exp(-l^2 / (2 sigma^2))      for l < r_cut     */

#define CSS_INT_NVE 0   /* velocity Verlet: v += dt/2m F; shift by dt v; F(x); v += dt/2m F */
#define CSS_INT_BD  1   /* lambda dr = dt F + sqrt(2 kT lambda dt) eta                      */
#define CSS_INT_ABP 2   /* dr = dt (v0 n + F / lambda); n rotated by sqrt(2 Dr dt) xi       */
#define CSS_INT_GD  3   /* steepest descent (Fig. 3 caption): dr = (dt / lambda) F, no noise */
#define CSS_INT_FIRE 4  /* FIRE minimiser (Bitzek et al. 2006): velocity Verlet with velocity
                           mixing and an adaptive step, see css_integrate_step             */

typedef struct css_ctx css_ctx;
typedef struct css_mesh css_mesh;
typedef struct css_parts css_parts;
typedef struct css_batch css_batch;

typedef struct {
    int32_t kind;          /* CSS_POT_*                                     */
    double eps, sigma;     /* energy scale, length scale                    */
    double r_cut;          /* U = 0 for l >= r_cut                          */
    double A;              /* Gaussian amplitude                            */
} css_potential;

typedef struct {
    int32_t kind;          /* CSS_INT_*                                     */
    double dt, kT, lambda; /* time step, temperature, friction              */
    double v0, Dr;         /* self-propulsion speed, rotational diffusion   */
    double mass;           /* particle mass (NVE)                           */
    double max_disp;       /* cap on |dr| per step (INFINITY: none)         */
} css_integrator;

/* ---------------------------------------------------------------- context
 * css_create: bind to CUDA device `device` and the cudaStream_t `stream`
 * (NULL: an owned non-blocking stream).  Fails with CSS_ERR_NO_DEVICE when no sm_103-class device
 * is present.  css_destroy frees the context's workspace (objects created
 * from it must be freed first). */
int css_create(css_ctx** out, int device, void* stream);
int css_destroy(css_ctx* ctx);
const char* css_last_error(const css_ctx* ctx);
/* Device-side counters of the last neighbour / force evaluation:
 * [0] sources, [1] windows created, [2] windows propagated, [3] pairs found (all summed
 * over the sources that completed), [4] sources deferred from the first pass to the
 * second (their patch overflowed the first pass's tables or window pool),
 * [5] workspace retries of the call. */
int css_last_counters(const css_ctx* ctx, int64_t out[6]);

/* ---------------------------------------------------------------- mesh (Sec. 2.2)
 * Upload a triangulated surface and precompute its intrinsic geometry on the
 * device: edges and adjacency, per-face planar layouts, half-edge frames and
 * the rigid maps between neighbouring faces, vertex angle sums, and the
 * pseudo-source vertices (boundary, flat or saddle: angle sum >= 2 pi - 1e-9).
 *   verts  nv x 3 doubles, faces nf x 3 int32 (row major), host or device.
 *   period NULL, or host pointer to {Lx, Ly}: x and y wrap with these periods
 *          and edge vectors use the minimum image.
 * Errors: CSS_ERR_INVALID_ARG (sizes, indices out of range, NaN),
 *         CSS_ERR_NONMANIFOLD (edge shared by >2 faces, inconsistent
 *         orientation, degenerate face). */
int css_mesh_upload(css_ctx* ctx, const double* verts, int64_t nv, const int32_t* faces,
                    int64_t nf, const double* period, css_mesh** out);
int css_mesh_free(css_mesh* mesh);
/* counts: nv, nf, number of undirected edges, number of pseudo-source vertices */
int css_mesh_counts(const css_mesh* mesh, int64_t out[4]);

/* ---------------------------------------------------------------- particles (Sec. 3)
 * A particle set bound to a mesh.  face: n int32; bary: n x 3 doubles summing
 * to 1 (each >= -1e-12); vel / orient: n x 3 world tangent vectors or NULL
 * (zero).  seed keys the Philox4x32-10 noise stream (counter = particle, step).
 * Errors: CSS_ERR_INVALID_ARG for a face index out of range, a barycentric
 * triple that does not sum to 1, or non-finite values. */
int css_particles_set(css_ctx* ctx, css_mesh* mesh, int64_t n, const int32_t* face,
                      const double* bary, const double* vel, const double* orient,
                      uint64_t seed, css_parts** out);
/* Copy state out (any pointer may be NULL): face n, bary n x 3, vel n x 3,
 * orient n x 3, force n x 3 (the last force evaluation), and the step counter. */
int css_particles_get(css_parts* parts, int32_t* face, double* bary, double* vel,
                      double* orient, double* force, int64_t* step);
/* Overwrite the state of an existing set (same n, same mesh) from host or device
 * buffers; any pointer may be NULL to keep that field.  No validation beyond the
 * face range is done on device inputs.  Used for checkpoint/resume and to feed a
 * simulation from host memory. */
int css_particles_update(css_parts* parts, const int32_t* face, const double* bary,
                         const double* vel, const double* orient);
/* Set the step counter (the Philox counter of the Brownian and active noise; what
 * css_particles_get returns as step).  With css_particles_set / css_particles_update of a
 * saved state and the same seed it resumes a stochastic run bit for bit.
 * CSS_ERR_INVALID_ARG for a negative step. */
int css_particles_set_step(css_parts* parts, int64_t step);
int css_particles_free(css_parts* parts);

/* ---------------------------------------------------------------- hot path
 * css_geodesic_neighbors (Sec. 3.1 "displacement"): every ordered pair (i, j),
 * i != j, with geodesic distance l_ij < r_c (r_c may be INFINITY: all pairs),
 * returned as CSR rows in source order with columns in increasing j:
 *   row_start n+1 int64, nbr_j int32, dist double, tangent 3 doubles per pair
 *   (unit initial direction at i of the geodesic towards j, world frame).
 * capacity is the length of nbr_j / dist (tangent holds 3 x capacity).  If it
 * is too small the call returns CSS_ERR_CAPACITY with *n_pairs set to the
 * needed count and writes nothing else.  Pairs with l_ij within 1e-9 r_c of
 * r_c may appear or not. */
int css_geodesic_neighbors(css_parts* parts, double r_c, int precision, int64_t capacity,
                           int64_t* n_pairs, int64_t* row_start, int32_t* nbr_j,
                           double* dist, double* tangent);

/* css_compute_forces (Sec. 3.1): F_i = sum_{l_ij < r_c} U'(l_ij) t_ij where t_ij is the
 * unit tangent at i towards j (so U' < 0 repels), and E_pot = 1/2 sum_ij U(l_ij).
 * forces: n x 3 doubles (world, in each particle's face plane) or NULL;
 * e_pot: one double or NULL.  The result is also stored in the particle set. */
int css_compute_forces(css_parts* parts, const css_potential* pot, double r_c, int precision,
                       double* forces, double* e_pot);

/* css_integrate_step (Sec. 2.1 + Sec. 3.2 "shift"): n_steps steps of the chosen
 * dynamics, each a complete pass: neighbour search within r_c, forces, and the
 * straightest face walk that moves every particle and parallel-transports its
 * velocity / orientation.  NVE reuses the force of the previous step (computed
 * on the first call).  noise: NULL (Philox stream) or a device/host array of
 * n_steps x n x 2 standard normals used instead (test mode).  The steps are
 * replayed from a captured CUDA graph when n_steps > 1 and noise is NULL.
 * e_pot (may be NULL) receives the potential energy of the last force pass.
 * CSS_INT_FIRE (no counterpart in the paper's text beyond the minimisations of Fig. 3):
 * each step computes P = sum F.v and the norms |v|, |F| over the set, mixes
 * v <- (1 - a) v + a |v| F / |F|, then after more than 5 steps in a row with P > 0 grows
 * the step (x 1.1, at most 10 x integ->dt) and shrinks a (x 0.99), while P <= 0 halves the
 * step, zeroes v and resets a = 0.1; then one velocity-Verlet step with the current step.
 * The state (step, a, count) lives on the device and starts from (integ->dt, 0.1, 0)
 * whenever the integrator parameters change or the particle state is replaced. */
int css_integrate_step(css_parts* parts, const css_potential* pot, const css_integrator* integ,
                       double r_c, int precision, int64_t n_steps, const double* noise,
                       double* e_pot);

/* css_trace_geodesics: the path of a pair as a polyline.  Path k is the straightest
 * geodesic (the face walk of css_integrate_step) from particle src[k] along the world
 * tangent tangent[3k..3k+2] (unit) for length[k]; with the tangent and distance of a pair
 * returned by css_geodesic_neighbors it is that pair's shortest path whenever the path
 * bends at no vertex (Sec. 2.2: shortest paths are straight in the unfolding of the faces
 * they cross) -- the end point then coincides with the neighbour, which callers can check
 * with end_face / end_bary.  Paths that bend at saddle, flat or boundary vertices are not
 * followed around the bend (the walk goes straight on); css_geodesic_paths returns those
 * paths with their bends.
 *   points   n_paths x max_points x 3 world positions: the start, every edge or vertex
 *            crossing, the end; unused entries are zero; max_points >= 2;
 *   n_points all points of each path (more than max_points when truncated);
 *   end_face, end_bary  the walk's end point.
 * Inputs and outputs may be host or device pointers.  Allocates temporaries and
 * synchronises.  CSS_ERR_INVALID_ARG for a source index out of range or a non-finite or
 * negative length or tangent. */
int css_trace_geodesics(css_parts* parts, int64_t n_paths, const int32_t* src, const double* tangent,
                        const double* length, int32_t max_points, double* points, int32_t* n_points,
                        int32_t* end_face, double* end_bary);

/* css_geodesic_paths (Sec. 2.2): the shortest path of each pair src[k] -> dst[k] as a
 * polyline, bends included.  A shortest path on the polyhedral surface is a chain of
 * straight legs (straight in the unfolding of the faces they cross) that meet at
 * pseudo-source vertices (boundary, flat or saddle vertices, where the window
 * propagation starts new windows).  This call runs the FP64 neighbour kernel for the
 * distinct sources with link recording: every vertex's table entry keeps the previous
 * node of its path (a pseudo-source vertex or the source), the direction towards it and
 * the leg's length, and every pair gets its chain of legs from the target back to the
 * source; each leg is then walked straight across the faces it crosses, passing straight
 * (angle pi on the side that holds it) through any vertex it meets on the way.
 *   points   n_pairs x max_points x 3 world positions (wrapped into the period on periodic
 *            meshes): the source particle, every edge or vertex crossing and every bend
 *            vertex in order, the target particle; unused entries are zero; max_points >= 2;
 *   n_points all points of each path (more than max_points: truncated, call again with
 *            more); 0 when l >= r_c;
 *   n_legs   straight legs of each path (1: no bend), 0 when l >= r_c;
 *   dist     l (INFINITY when l >= r_c);
 *   gap      the largest distance between where a leg's walk ends and the node it must
 *            reach (a check of the result; rounding size).
 * r_c may be INFINITY.  Inputs and outputs may be host or device pointers.  Allocates
 * temporaries and synchronises.  CSS_ERR_INVALID_ARG for an index out of range or
 * src[k] == dst[k]; CSS_ERR_QUEUE_OVERFLOW when the window pool cannot grow enough;
 * CSS_ERR_ITER_LIMIT when a path has more than 32 legs or a leg walk fails. */
int css_geodesic_paths(css_parts* parts, double r_c, int64_t n_pairs, const int32_t* src, const int32_t* dst,
                       int32_t max_points, double* points, int32_t* n_points, int32_t* n_legs, double* dist,
                       double* gap);

/* css_vhm_neighbors: approximate geodesic distances and initial tangents for every ordered
 * pair (i, j), i != j, with the approximate distance below r_c (INFINITY: all pairs), in the
 * layout of css_geodesic_neighbors.  This is the approximate alternative the paper names
 * beside exact window propagation (Sec. 2.2: the vector heat method, O(h) error on a mesh of
 * spacing h; Sec. 5).  Per source particle q, FP64, on the whole mesh:
 *   (M + t L) u = u0       one backward-Euler heat step (L cotan Laplacian, M lumped mass,
 *                          t = t_factor * h^2, h the mean edge length, u0 = q's barycentrics
 *                          on its face's corners);
 *   (M + t Lc) Y = Y0      the same step for tangent vectors (Lc the connection Laplacian over
 *                          vertex frames whose corner angles are scaled to close up; Y0 = the
 *                          source face's x-axis): H = Y / |Y| is that axis transported;
 *   L phi = -div(-grad u / |grad u|)   (right-hand side made mean-free), phi(q) = 0;
 * then l_ij = phi(x_j) (linear interpolation) and t_ij = the source face's x-axis turned by the
 * angle of grad phi against H at x_j.  The heat steps are solved by Gauss-Seidel sweeps over
 * a colouring of the vertex graph (convergent on any mesh: the systems are symmetric positive
 * definite) until no entry changes by more than
 * 1e-14 of the terms it is summed from (entries below 1e-290, i.e. farther than about
 * 660 sqrt(t) from the source, have no relative accuracy left), the Poisson step by
 * conjugate gradients to 1e-14 of the preconditioned residual.  t_factor > 0 (1: t = h^2).
 * Allocates a workspace and synchronises.  css_last_counters then holds: sources, the
 * largest heat-sweep count of a batch, conjugate-gradient iterations (summed over batches),
 * pairs, batches, sources per batch.
 * Errors: CSS_ERR_INVALID_ARG (t_factor <= 0 or not finite, r_c NaN or <= 0),
 * CSS_ERR_CAPACITY (as css_geodesic_neighbors), CSS_ERR_NONMANIFOLD (a vertex whose faces are
 * not one disk or half-disk), CSS_ERR_ITER_LIMIT (a solve did not converge in 50000 steps). */
int css_vhm_neighbors(css_parts* parts, double r_c, double t_factor, int64_t capacity, int64_t* n_pairs,
                      int64_t* row_start, int32_t* nbr_j, double* dist, double* tangent);

/* ---------------------------------------------------------------- batched form
 * Many independent particle sets (each on its own mesh) advanced together: the
 * neighbour/force work of all sets runs in one persistent launch per step whose
 * warps pull (set, source) items from a device work queue (sets with more particles
 * first), moves and face bucketing of all sets run as single launches, and one step is
 * captured into a CUDA graph (kept while the parameters stay the same) and replayed.
 * The sets must come from the same context; they share pot/integ/r_c.  CSS_INT_FIRE is
 * per set (its norms are over one set) and is rejected here with CSS_ERR_INVALID_ARG. */
int css_batch_create(css_ctx* ctx, css_parts* const* parts, int32_t n_sets, css_batch** out);
int css_batch_step(css_batch* batch, const css_potential* pot, const css_integrator* integ,
                   double r_c, int precision, int64_t n_steps);
int css_batch_free(css_batch* batch);

/* ---------------------------------------------------------------- allocation-free forces
 * css_compute_forces_noalloc has no counterpart in the paper.  It is for callers that
 * cannot allocate device memory where they evaluate forces (inside a host callback, in
 * a framework that forbids allocation on its hot path, or where the device footprint
 * must stay fixed after start-up).  It computes the same forces and energy as
 * css_compute_forces, for particles given directly as device arrays, and calls no
 * cudaMalloc, cudaFree or allocating library routine: its scratch is one fixed device
 * array of about 59 MB that every GPU loading this library holds until exit.
 *   mesh     uploaded beforehand with css_mesh_upload (that call allocates); the call runs
 *            on the device of the mesh's context, whatever device is current, and puts
 *            the caller's current device back before it returns;
 *   face     device int32[n]; bary device double[n x 3]; forces device double[n x 3];
 *   e_pot    device double[1] or NULL (zeroed, then summed into);
 *   stream   cudaStream_t of the mesh's device to run on (NULL: that device's legacy
 *            default stream); the call first makes it wait for the work queued on the
 *            context's stream (an update or a step writing face / bary), and synchronises
 *            it to read the status.
 * The particle arrays are checked on the device before any kernel indexes with them: a
 * face outside [0, nf) or a barycentric triple that is not finite, has an entry below
 * -1e-12 or does not sum to 1 within 1e-9 gives CSS_ERR_INVALID_ARG, as does a stream of
 * another device.
 * Limits: n <= 262144 particles, at most 1048576 faces, 2048 windows per source and
 * warp; beyond them it returns CSS_ERR_CAPACITY (sizes) or CSS_ERR_QUEUE_OVERFLOW (a
 * source needing more windows), and css_compute_forces should be used instead; a device
 * loop cap gives CSS_ERR_ITER_LIMIT.
 * The first call on a device looks up the array's device address (set-up): make it
 * before any stream capture.  Every call shares the array, which keeps the previous
 * call's contents, so calls that overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller. */
int css_compute_forces_noalloc(const css_mesh* mesh, int64_t n, const int32_t* face,
                               const double* bary, const css_potential* pot, double r_c,
                               int precision, double* forces, double* e_pot, void* stream);

/* ---------------------------------------------------------------- measurement
 * css_last_kernel_ms: device time (ms) between CUDA events recorded on the context
 * stream immediately before the first and after the second pass of the last
 * neighbour/force evaluation (inside captured graphs too).  CSS_ERR_INVALID_ARG before
 * any launch.
 * css_fma_peak: measured dense FMA throughput (flop/s, 2 per FMA) of this GPU's
 * FP32 or FP64 pipes, from an FMA-chain kernel filling every SM; it has no
 * counterpart in the paper and serves as the ALU roofline denominator. */
int css_last_kernel_ms(css_ctx* ctx, double* ms);
int css_fma_peak(css_ctx* ctx, int precision, double* flops_per_s);

/* ---------------------------------------------------------------- tuning
 * Launch shape of the neighbour/force evaluation (no counterpart in the paper, whose
 * method runs one source per CPU process).  Every source runs in a first pass: one
 * warp per source, per-warp hash tables (edges, pseudo-source vertices, faces) in
 * shared memory and a window pool in global memory.  A source whose patch overflows
 * them is deferred, and a second pass re-runs the deferred sources with global-memory
 * tables and a larger pool on fewer warps.  Results do not depend on the shape.
 *   warps_per_cta      first pass, 1..8
 *   ctas_per_sm        first pass resident CTAs per SM, 0 = as many as fit, else a cap
 *                      (fewer resident warps keep more of each warp's pool in L2)
 *   tile               work items (sources) a warp claims per atomic, 1..64
 *   shared_scale       first-pass table size, 0 (global tables), 1, 2, 4 or 8 times
 *                      512 edges / 256 vertices / 512 faces per warp
 *   window_capacity    first-pass windows per warp, 64..2^20 (rounded up to 2^k)
 *   window_capacity2   second-pass windows per warp (grown on overflow)
 *   warps2_per_sm      second-pass warps per SM, 1..8
 *   occupancy          first-pass register budget: 1 = up to 255 registers a thread (at
 *                      most 8 resident warps per SM, no spills), 2 = at most 128 (twice
 *                      the resident warps, some spills to local memory)
 *   table_capacity     first pass with global tables (shared_scale 0): edge and face table
 *                      slots per warp, vertex slots half of it (rounded up to 2^k, 64..2^20);
 *                      0 = tied to window_capacity.  Tables sized for the patches of the
 *                      workload keep each source's entries on few cache lines; a source
 *                      that overflows them is deferred to the second pass
 *   team               0: one warp per source; 1: all warps of a CTA (warps_per_cta >= 2) work
 *                      on one source together -- each wave unfolds up to 32 x warps_per_cta
 *                      windows and the insertions are spread over the warps by edge and vertex
 *                      id -- for sets with fewer sources than resident warps
 * css_set_launch fails with CSS_ERR_INVALID_ARG when a value is out of range or the
 * shape's shared memory does not fit an SM.  Until a shape is set or tuned, a context
 * starts from {4, 0, 1, 1, 2048, 16384, 2, 1, 0, 0} and adapts by itself: after an evaluation
 * that deferred more than a quarter of its sources it switches the first pass to global
 * tables with a four times larger pool (up to 2^17 windows). */
typedef struct css_launch {
    int32_t warps_per_cta, ctas_per_sm, tile, shared_scale;
    int32_t window_capacity, window_capacity2, warps2_per_sm, occupancy;
    int32_t table_capacity;
    int32_t team;
} css_launch;
int css_set_launch(css_ctx* ctx, const css_launch* launch);
int css_get_launch(const css_ctx* ctx, css_launch* launch);

/* Autotuner: times the force evaluation of the given sets (one persistent launch over
 * all their sources, as the batched form runs it) under candidate launch shapes --
 * shared_scale x warps_per_cta x ctas_per_sm, with a first-pass pool of 2048 windows
 * times the scale (8192 for global tables, whose tables are tried both tied to the pool
 * and at 4096 slots), and four times that pool where more than 1 % of the sources were
 * deferred, then occupancy 2 with 4 or 8 warps per CTA (global tables with pools of 8192
 * and 32768 windows, tables tied or at 4096 slots, and the best pick's tables), then, when the
 * sources sampled are fewer than four times 8 warps per SM, the team form (shared tables at
 * scale 1 or 4 or global tables x 2, 4, 8 warps per CTA x occupancy 1, 2, pools grown four and
 * sixteen times while sources are deferred), then the tile on the best (not for a
 * team) -- and keeps the fastest in the context.  Each candidate runs `reps` times (>= 1) after one
 * untimed run; `sample` > 0 restricts every run to about that many sources spread over
 * the sets (0: all).  best (may be NULL) receives the chosen shape and best_ms its
 * time.  Particle states are unchanged; stored forces are marked stale.  Synchronises. */
int css_autotune(css_ctx* ctx, css_parts* const* sets, int32_t n_sets, const css_potential* pot, double r_c,
                 int precision, int32_t reps, int64_t sample, css_launch* best, double* best_ms);

#ifdef __cplusplus
}
#endif
#endif /* CSS_H */
